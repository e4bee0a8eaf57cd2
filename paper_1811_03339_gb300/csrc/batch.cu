// Batched assembly and solve of many meshes of uneven size (not in the paper: the paper
// assembles one mesh at a time).  One launch walks every Gauss-point line of every mesh;
// contraction, load vector and factorisation of each mesh run on internal streams so
// that small meshes overlap; each refinement sweep solves all meshes in one batched
// block-step triangular solve and checks all residuals with a single host wait.
//
// The assembly and factorisation of the whole batch (walk, contractions, load vectors,
// factorisations: everything before the first refinement sweep) is captured as one CUDA
// graph the second time a run has the same orders, coefficients, precision, column count and
// right-hand-side arrays, and replayed as one graph launch from then on (the first run goes
// eagerly: it makes the allocations, the tile tuner's timings and the factorisation's side
// streams that a capture must not make).  The refinement sweeps stay host-driven: each one
// checks the residuals before the next.
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

struct Batch {
    std::vector<Mesh *> ms;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;   // one per internal stream
    cudaEvent_t fork = nullptr;
    BatchWalkScratch ws;
    BatchTrsmDesc *d_tdesc = nullptr, *h_tdesc = nullptr;
    int max_nblk = 0;
    // per-mesh run buffers, kept across runs (a captured graph refers to their addresses):
    // load vector b, residual r, A u (column-major, n_dof x nrhs) and the FP32 correction
    std::vector<double *> bv, rv, auv;
    std::vector<float *> r32;
    int nrhs_cap = 0;
    // the captured assembly + factorisation and what it was captured for
    cudaGraphExec_t exec = nullptr;
    // the capture runs on a private stream (the caller's may be the legacy stream, which
    // cannot be captured); it starts after the work enqueued so far on the caller's stream
    cudaStream_t cap = nullptr;
    cudaEvent_t cap_in = nullptr;
    std::vector<double> key_ak;          // alpha, K
    std::vector<const double *> key_f;   // right-hand-side arrays
    int key_prec = -1, key_nrhs = 0;
    int runs = 0;                        // eager runs so far
    int graph_launches = 0;              // replays so far
};

static void free_run_buffers(Batch *b) {
    for (double *p : b->bv) cudaFree(p);
    for (double *p : b->rv) cudaFree(p);
    for (double *p : b->auv) cudaFree(p);
    for (float *p : b->r32) cudaFree(p);
    b->bv.clear();
    b->rv.clear();
    b->auv.clear();
    b->r32.clear();
    b->nrhs_cap = 0;
}

static void batch_destroy(Batch *b) {
    if (!b) return;
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    free_run_buffers(b);
    for (Mesh *m : b->ms) fem3_mesh_free(reinterpret_cast<fem3_mesh>(m));
    for (cudaEvent_t e : b->done) cudaEventDestroy(e);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap_in) cudaEventDestroy(b->cap_in);
    cudaFree(b->ws.d_desc);
    cudaFreeHost(b->ws.h_desc);
    cudaFree(b->d_tdesc);
    cudaFreeHost(b->h_tdesc);
    delete b;
}

// every internal stream waits for the work enqueued so far on `s`
static int fork_to(Batch *b, cudaStream_t s) {
    FEM3_CUDA(cudaEventRecord(b->fork, s));
    for (cudaStream_t t : b->streams) FEM3_CUDA(cudaStreamWaitEvent(t, b->fork, 0));
    return FEM3_OK;
}
// `s` waits for the work enqueued so far on every internal stream
static int join_to(Batch *b, cudaStream_t s) {
    for (size_t k = 0; k < b->streams.size(); k++) {
        FEM3_CUDA(cudaEventRecord(b->done[k], b->streams[k]));
        FEM3_CUDA(cudaStreamWaitEvent(s, b->done[k], 0));
    }
    return FEM3_OK;
}

__global__ void k_copy_to_f32(const double *__restrict__ a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_add_f32(const float *__restrict__ d, double *u, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] += (double)d[i];
}
__global__ void k_resid_cols(const double *__restrict__ b, const double *__restrict__ Au, int64_t n,
                             double *r, double *norms) {
    const int c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0, bb = 0;
    if (i < n) {
        const int64_t k = (int64_t)c * n + i;
        const double v = b[k] - Au[k];
        r[k] = v;
        rr = v * v;
        bb = b[k] * b[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&norms[2 * c], rr);
        atomicAdd(&norms[2 * c + 1], bb);
    }
}

static inline unsigned blocks(int64_t n) { return (unsigned)(n > 0 ? (n + 255) / 256 : 1); }

static int check_mesh(Mesh *m, int i) {
    int32_t e[ERR_COUNT];
    FEM3_TRY(read_errors(m, e));
    const std::string who = "mesh " + std::to_string(i) + ": ";
    if (e[ERR_WALK]) return set_error(FEM3_E_WALK, who + "a path walk exceeded its step cap");
    if (e[ERR_TEMPLATE]) return set_error(FEM3_E_TEMPLATE, who + "table update outside the template");
    if (e[ERR_NOT_SPD]) {
        cudaMemsetAsync(m->err + ERR_NOT_SPD, 0, sizeof(int32_t), m->stream);
        return set_error(FEM3_E_NOT_SPD, who + "non-positive pivot at column " +
                                             std::to_string(e[ERR_NOT_SPD] - 1));
    }
    if (e[ERR_TC] || e[ERR_SOLVE] || e[ERR_CHOL]) return set_error(FEM3_E_CUDA, who + "a bounded wait expired");
    return FEM3_OK;
}

}  // namespace fem3

using namespace fem3;

extern "C" {

int fem3_batch_create(int n_meshes, const double *const *verts, const int64_t *n_nodes,
                      const int32_t *const *tets, const int64_t *n_tets, const fem3_options *opt,
                      void *stream, fem3_batch *out) {
    if (!out || n_meshes < 1 || !verts || !n_nodes || !tets || !n_tets)
        return set_error(FEM3_E_ARG, "bad argument");
    *out = nullptr;
    Batch *b = new Batch();
    for (int i = 0; i < n_meshes; i++) {
        fem3_mesh h = nullptr;
        int st = fem3_mesh_upload(verts[i], n_nodes[i], tets[i], n_tets[i], opt, stream, &h);
        if (st != FEM3_OK) {
            batch_destroy(b);
            return st;
        }
        b->ms.push_back(reinterpret_cast<Mesh *>(h));
    }
    const int ns = std::min(n_meshes, 8);
    for (int k = 0; k < ns; k++) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            batch_destroy(b);
            return cuda_error(cudaGetLastError(), "stream/event creation");
        }
        b->streams.push_back(s);
        b->done.push_back(e);
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->cap_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMalloc(&b->d_tdesc, sizeof(BatchTrsmDesc) * n_meshes) != cudaSuccess ||
        cudaMallocHost(&b->h_tdesc, sizeof(BatchTrsmDesc) * n_meshes) != cudaSuccess) {
        batch_destroy(b);
        return cuda_error(cudaGetLastError(), "batch allocation");
    }
    for (Mesh *m : b->ms) b->max_nblk = std::max<int>(b->max_nblk, (int)((m->n_dof + 63) / 64));
    *out = reinterpret_cast<fem3_batch>(b);
    return FEM3_OK;
}

int fem3_batch_mesh(fem3_batch hb, int i, fem3_mesh *out) {
    Batch *b = reinterpret_cast<Batch *>(hb);
    if (!b || !out || i < 0 || i >= (int)b->ms.size()) return set_error(FEM3_E_ARG, "bad argument");
    *out = reinterpret_cast<fem3_mesh>(b->ms[i]);
    return FEM3_OK;
}

int fem3_batch_run(fem3_batch hb, const double *alpha, const double *K, int precision,
                   const double *const *f, int nrhs, double tol, int max_iter, double *const *u,
                   int *iters, double *resid, void *stream) {
    Batch *b = reinterpret_cast<Batch *>(hb);
    if (!b || !alpha || !K || !f || !u || nrhs < 1 || nrhs > 16)
        return set_error(FEM3_E_ARG, "bad argument (1 <= nrhs <= 16)");
    if (precision != FEM3_FP64 && precision != FEM3_TF32X3 && precision != FEM3_FP32 &&
        precision != FEM3_BF16X3)
        return set_error(FEM3_E_ARG, "unknown precision");
    const int n = (int)b->ms.size();
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
    for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            if (!(alpha[3 * i + a] > 1.0 && alpha[3 * i + a] <= 2.0))
                return set_error(FEM3_E_ARG, "alpha must lie in (1, 2]");
            if (!(K[3 * i + a] > 0.0)) return set_error(FEM3_E_ARG, "K must be positive");
        }
    if (max_iter <= 0) max_iter = 50;
    const bool fp64 = precision == FEM3_FP64;

    // host-side state of every mesh for this run (the refinement reads it)
    for (int i = 0; i < n; i++) {
        Mesh *m = b->ms[i];
        m->stream = cs;
        const int64_t nd = m->n_dof;
        if (fp64 && !m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, std::max<int64_t>(1, nd * nd)));
        if (!fp64 && !m->A32) FEM3_TRY(dev_alloc_t(m, &m->A32, std::max<int64_t>(1, nd * nd)));
        for (int a = 0; a < 3; a++) {
            m->alpha[a] = alpha[3 * i + a];
            m->K[a] = K[3 * i + a];
            m->s[a] = 1.0 / (2.0 * cos(M_PI * m->alpha[a] / 2.0));
            m->sK[a] = m->s[a] * m->K[a];
        }
        m->precision = precision;
        m->factored = false;
        m->ap_ready = false;
    }
    // run buffers for nrhs columns (kept across runs)
    if (b->nrhs_cap < nrhs) {
        for (cudaStream_t t : b->streams) FEM3_CUDA(cudaStreamSynchronize(t));
        FEM3_CUDA(cudaStreamSynchronize(cs));
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        free_run_buffers(b);
        b->bv.assign(n, nullptr);
        b->rv.assign(n, nullptr);
        b->auv.assign(n, nullptr);
        b->r32.assign(n, nullptr);
        for (int i = 0; i < n; i++) {
            const size_t nn = (size_t)std::max<int64_t>(1, b->ms[i]->n_dof * nrhs);
            if (cudaMalloc((void **)&b->bv[i], sizeof(double) * nn) != cudaSuccess ||
                cudaMalloc((void **)&b->rv[i], sizeof(double) * nn) != cudaSuccess ||
                cudaMalloc((void **)&b->auv[i], sizeof(double) * nn) != cudaSuccess ||
                cudaMalloc((void **)&b->r32[i], sizeof(float) * nn) != cudaSuccess)
                return cuda_error(cudaGetLastError(), "cudaMalloc (batch run buffers)");
        }
        b->nrhs_cap = nrhs;
    }
    std::vector<double *> &bv = b->bv, &rv = b->rv, &auv = b->auv;
    std::vector<float *> &r32 = b->r32;

    // 1 + 2: walk of every line of every mesh (one launch on the caller's stream), then per
    // mesh on the internal streams contraction, load vector and factorisation; replayed
    // from the captured graph when the run matches the one it was captured for
    std::vector<double> ak(alpha, alpha + 3 * n);
    ak.insert(ak.end(), K, K + 3 * n);
    std::vector<const double *> fk(f, f + n);
    const bool same = b->exec && b->key_prec == precision && b->key_nrhs == nrhs &&
                      b->key_ak == ak && b->key_f == fk;
    auto enqueue_assembly = [&](cudaStream_t os) -> int {
        FEM3_TRY(walk_tables_batch(b->ms.data(), n, alpha, os, &b->ws));
        FEM3_TRY(fork_to(b, os));
        for (int i = 0; i < n; i++) {
            Mesh *m = b->ms[i];
            m->stream = b->streams[i % b->streams.size()];
            if (m->n_dof == 0) continue;
            if (precision == FEM3_TF32X3 || precision == FEM3_BF16X3)
                FEM3_TRY(contract_tc(m, precision == FEM3_BF16X3));
            else
                FEM3_TRY(contract(m, precision));
            FEM3_TRY(load_vector(m, f[i], nrhs, bv[i]));
            FEM3_TRY(factor(m));
        }
        FEM3_TRY(join_to(b, os));
        return FEM3_OK;
    };
    int st = FEM3_OK;
    if (same) {
        FEM3_CUDA(cudaGraphLaunch(b->exec, cs));
        b->graph_launches++;
        // the replayed contraction wrote the apply operands, as the captured one did
        const bool tc = precision == FEM3_TF32X3 || precision == FEM3_BF16X3;
        for (Mesh *m : b->ms) m->ap_ready = tc && m->n_dof > 0;
    } else if (b->runs >= 1) {
        // capture the assembly + factorisation; on any failure discard it and run eagerly
        if (b->exec) {
            FEM3_CUDA(cudaStreamSynchronize(cs));
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        bool captured = false;
        FEM3_CUDA(cudaEventRecord(b->cap_in, cs));
        FEM3_CUDA(cudaStreamWaitEvent(b->cap, b->cap_in, 0));
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int cst = enqueue_assembly(b->cap);
            const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
            if (cst == FEM3_OK && ce == cudaSuccess && g &&
                cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                captured = true;
                b->key_prec = precision;
                b->key_nrhs = nrhs;
                b->key_ak = ak;
                b->key_f = fk;
            }
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
        if (captured) {
            FEM3_CUDA(cudaGraphLaunch(b->exec, cs));
            b->graph_launches++;
        } else {
            b->exec = nullptr;
            st = enqueue_assembly(cs);
        }
    } else {
        st = enqueue_assembly(cs);
        b->runs++;
    }
    // the first correction starts from u = 0: the residual is b
    if (st == FEM3_OK) st = fork_to(b, cs);
    for (int i = 0; i < n && st == FEM3_OK; i++) {
        Mesh *m = b->ms[i];
        m->stream = b->streams[i % b->streams.size()];
        if (m->n_dof == 0) continue;
        m->factored = true;
        FEM3_CUDA(cudaMemcpyAsync(rv[i], bv[i], sizeof(double) * m->n_dof * nrhs,
                                  cudaMemcpyDeviceToDevice, m->stream));
        FEM3_CUDA(cudaMemsetAsync(u[i], 0, sizeof(double) * m->n_dof * nrhs, m->stream));
    }

    // 3. refinement (FP64: a single direct sweep)
    std::vector<int> it(n, 0);
    std::vector<double> worst(n, 0.0);
    std::vector<char> active(n, 1);
    for (int i = 0; i < n; i++) active[i] = b->ms[i]->n_dof > 0;
    BatchTrsmDesc *hd = b->h_tdesc;
    int sweep = 0;
    while (st == FEM3_OK) {
        // right-hand sides of the triangular solves
        int n_active = 0;
        for (int i = 0; i < n; i++) {
            Mesh *m = b->ms[i];
            hd[i] = BatchTrsmDesc{fp64 ? (const void *)m->A64 : (const void *)m->A32, m->dinv,
                                  fp64 ? (void *)u[i] : (void *)r32[i], m->n_dof,
                                  (int)((m->n_dof + 63) / 64), active[i] ? 1 : 0};
            if (!active[i]) continue;
            n_active++;
            const int64_t nn = m->n_dof * nrhs;
            if (fp64) {
                FEM3_CUDA(cudaMemcpyAsync(u[i], bv[i], sizeof(double) * nn, cudaMemcpyDeviceToDevice,
                                          m->stream));
            } else {
                k_copy_to_f32<<<blocks(nn), 256, 0, m->stream>>>(rv[i], r32[i], nn);
                note_launch(m);
            }
        }
        if (n_active == 0) break;
        FEM3_TRY(join_to(b, cs));
        FEM3_CUDA(cudaMemcpyAsync(b->d_tdesc, hd, sizeof(BatchTrsmDesc) * n, cudaMemcpyHostToDevice, cs));
        FEM3_TRY(trsm_batch(b->d_tdesc, n, b->max_nblk, nrhs, fp64, cs));
        FEM3_TRY(fork_to(b, cs));
        sweep++;
        if (fp64) break;
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            Mesh *m = b->ms[i];
            const int64_t nn = m->n_dof * nrhs;
            k_add_f32<<<blocks(nn), 256, 0, m->stream>>>(r32[i], u[i], nn);
            note_launch(m);
            if ((st = apply_multi(m, u[i], nrhs, auv[i])) != FEM3_OK) break;
            FEM3_CUDA(cudaMemsetAsync(m->norms, 0, sizeof(double) * 2 * nrhs, m->stream));
            k_resid_cols<<<dim3(blocks(m->n_dof), nrhs), 256, 0, m->stream>>>(bv[i], auv[i], m->n_dof,
                                                                           rv[i], m->norms);
            note_launch(m);
            FEM3_CUDA(cudaMemcpyAsync(m->h_norms, m->norms, sizeof(double) * 2 * nrhs,
                                      cudaMemcpyDeviceToHost, m->stream));
        }
        for (cudaStream_t t : b->streams) FEM3_CUDA(cudaStreamSynchronize(t));
        for (int i = 0; i < n; i++) {
            if (!active[i]) continue;
            Mesh *m = b->ms[i];
            double w = 0;
            for (int c = 0; c < nrhs; c++) {
                const double rel = m->h_norms[2 * c + 1] > 0 ? sqrt(m->h_norms[2 * c] / m->h_norms[2 * c + 1]) : 0.0;
                w = rel == rel ? std::max(w, rel) : INFINITY;
            }
            worst[i] = w;
            it[i] = sweep;
            if (w <= tol || sweep >= max_iter || !(w < INFINITY)) active[i] = 0;
        }
    }

    // 4. join into the caller's stream, report
    FEM3_TRY(join_to(b, cs));
    if (st != FEM3_OK) return st;
    int bad = FEM3_OK;
    for (int i = 0; i < n; i++) {
        Mesh *m = b->ms[i];
        m->stream = cs;
        if (iters) iters[i] = fp64 ? 0 : it[i];
        if (resid) resid[i] = worst[i];
        int e = check_mesh(m, i);
        if (e != FEM3_OK && bad == FEM3_OK) bad = e;
        if (!fp64 && m->n_dof > 0 && !(worst[i] <= tol) && bad == FEM3_OK)
            bad = set_error(FEM3_E_NO_CONVERGE, "mesh " + std::to_string(i) +
                                                    ": iterative refinement did not converge");
    }
    return bad;
}

int fem3_batch_graph_launches(fem3_batch hb, int64_t *n) {
    Batch *b = reinterpret_cast<Batch *>(hb);
    if (!b || !n) return set_error(FEM3_E_ARG, "bad argument");
    *n = b->graph_launches;
    return FEM3_OK;
}

void fem3_batch_free(fem3_batch hb) { batch_destroy(reinterpret_cast<Batch *>(hb)); }

}  // extern "C"
