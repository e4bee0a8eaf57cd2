// C ABI entry points of libfem3 (declared in include/fem3.h).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_error(cudaError_t e, const char *where) {
    int code = (e == cudaErrorMemoryAllocation) ? FEM3_E_OOM : FEM3_E_CUDA;
    return set_error(code, std::string(where) + ": " + cudaGetErrorString(e));
}

// Device memory of a mesh lives until the mesh is freed.  Requests up to kArenaMax bytes
// are carved (256-byte aligned) from 64 MB stream-ordered chunks, so a mesh makes a few
// allocator calls instead of one per array; larger ones get their own allocation.
constexpr size_t kArenaChunk = size_t(64) << 20, kArenaMax = size_t(16) << 20;

static int raw_alloc(Mesh *m, void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMallocAsync(p, bytes, m->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_error(e, "cudaMallocAsync");
    }
    m->allocs.push_back(*p);
    return FEM3_OK;
}

int dev_alloc(Mesh *m, void **p, size_t bytes) {
    bytes = (std::max<size_t>(bytes, 1) + 255) & ~size_t(255);
    if (bytes > kArenaMax) return raw_alloc(m, p, bytes);
    if (!m->arena || m->arena_used + bytes > m->arena_size) {
        void *c;
        FEM3_TRY(raw_alloc(m, &c, kArenaChunk));
        m->arena = static_cast<char *>(c);
        m->arena_size = kArenaChunk;
        m->arena_used = 0;
    }
    *p = m->arena + m->arena_used;
    m->arena_used += bytes;
    return FEM3_OK;
}

void dev_free_all(Mesh *m) {
    for (void *p : m->allocs) cudaFreeAsync(p, m->stream);
    m->allocs.clear();
    m->arena = nullptr;
    m->arena_size = m->arena_used = 0;
}

// Pinned 1 KB host blocks for the small device-to-host reads of a mesh, kept for the
// life of the process (pinned allocation and release are slow and release synchronises).
static std::mutex g_pin_mu;
static std::vector<double *> g_pin_free;
static double *pinned_block() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        double *c = nullptr;
        if (cudaMallocHost(&c, 64 * 128 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = 0; i < 64; i++) g_pin_free.push_back(c + 128 * i);
    }
    double *p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}
static void pinned_release(double *p) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void stage_begin(Mesh *m, int stage) {
    if (m->profile) cudaEventRecord(m->ev[2 * stage], m->stream);
}
void stage_end(Mesh *m, int stage) {
    if (m->profile) cudaEventRecord(m->ev[2 * stage + 1], m->stream);
}
void stage_collect(Mesh *m) {
    if (!m->profile) return;
    cudaStreamSynchronize(m->stream);
    for (int k = 0; k < 7; k++) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m->ev[2 * k], m->ev[2 * k + 1]) == cudaSuccess)
            m->stage_ms[k] = ms;
        else
            cudaGetLastError();
    }
    for (size_t i = 0; i < m->kc_used; i++) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, m->kc_ev[2 * i], m->kc_ev[2 * i + 1]) == cudaSuccess) {
            m->kc_ms[m->kc_cls[i]] += ms;
            m->kc_n[m->kc_cls[i]]++;
        } else {
            cudaGetLastError();
        }
    }
    m->kc_used = 0;
}

void kc_begin(Mesh *m, int cls) {
    if (!m->profile) return;
    while (m->kc_ev.size() < 2 * (m->kc_used + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        m->kc_ev.push_back(e);
    }
    if (m->kc_cls.size() < m->kc_used + 1) m->kc_cls.resize(m->kc_used + 1);
    m->kc_cls[m->kc_used] = cls;
    cudaEventRecord(m->kc_ev[2 * m->kc_used], m->stream);
}

void kc_end(Mesh *m, int cls) {
    if (!m->profile || m->kc_ev.size() < 2 * (m->kc_used + 1) || m->kc_cls[m->kc_used] != cls)
        return;
    cudaEventRecord(m->kc_ev[2 * m->kc_used + 1], m->stream);
    m->kc_used++;
}

void kc_reset(Mesh *m) {
    m->kc_used = 0;
    for (int k = 0; k < 8; k++) {
        m->kc_ms[k] = 0.f;
        m->kc_n[k] = 0;
    }
}

int read_errors(Mesh *m, int32_t *h_err) {
    FEM3_CUDA(cudaMemcpyAsync(h_err, m->err, sizeof(int32_t) * ERR_COUNT, cudaMemcpyDeviceToHost,
                              m->stream));
    FEM3_CUDA(cudaStreamSynchronize(m->stream));
    return FEM3_OK;
}

static int check_errors(Mesh *m) {
    int32_t e[ERR_COUNT];
    FEM3_TRY(read_errors(m, e));
    if (e[ERR_WALK])
        return set_error(FEM3_E_WALK, std::to_string(e[ERR_WALK]) +
                                          " path walks exceeded the step cap or found no exit");
    if (e[ERR_TEMPLATE])
        return set_error(FEM3_E_TEMPLATE, std::to_string(e[ERR_TEMPLATE]) +
                                              " table updates fell outside the bin template");
    if (e[ERR_NOT_SPD]) {
        int col = e[ERR_NOT_SPD] - 1;
        cudaMemsetAsync(m->err + ERR_NOT_SPD, 0, sizeof(int32_t), m->stream);
        return set_error(FEM3_E_NOT_SPD,
                         "non-positive pivot in Cholesky at column " + std::to_string(col));
    }
    if (e[ERR_MESH] || e[ERR_FACE]) return set_error(FEM3_E_MESH, "mesh error");
    if (e[ERR_SOLVE])
        return set_error(FEM3_E_CUDA, "a triangular-solve wait gave up (bounded wait expired)");
    if (e[ERR_TC])
        return set_error(FEM3_E_CUDA, "a tensor-core contraction wait gave up (bounded wait expired)");
    if (e[ERR_CHOL])
        return set_error(FEM3_E_CUDA, "a factorisation wait gave up (bounded wait expired)");
    return FEM3_OK;
}

// Copy a host or device array into a device buffer owned by the mesh (or return the
// device pointer itself).
static int to_device(Mesh *m, const void *src, size_t bytes, const void **dst, void **owned) {
    *owned = nullptr;
    if (is_device_ptr(src)) {
        *dst = src;
        return FEM3_OK;
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, m->stream);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
    e = cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(p, m->stream);
        return cuda_error(e, "cudaMemcpyAsync");
    }
    *dst = p;
    *owned = p;
    return FEM3_OK;
}

}  // namespace fem3

using namespace fem3;

extern "C" {

int fem3_last_error(char *buf, size_t len) {
    if (!buf || len == 0) return FEM3_E_ARG;
    snprintf(buf, len, "%s", g_last_error.c_str());
    return FEM3_OK;
}

void fem3_mesh_free(fem3_mesh h) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m) return;
    dev_free_all(m);
    cudaStreamSynchronize(m->stream);
    if (m->h_norms) pinned_release(m->h_norms);
    if (m->ev_made)
        for (int k = 0; k < 16; k++) cudaEventDestroy(m->ev[k]);
    for (cudaEvent_t e : m->kc_ev) cudaEventDestroy(e);
    delete m;
}

int fem3_mesh_upload(const double *verts, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                     const fem3_options *opt, void *stream, fem3_mesh *out) {
    if (!verts || !tets || !out) return set_error(FEM3_E_ARG, "null argument");
    *out = nullptr;
    if (n_nodes < 4 || n_nodes >= (1ll << 21) || n_tets < 1 || n_tets >= (1ll << 29))
        return set_error(FEM3_E_ARG, "mesh size out of range (4 <= n_nodes < 2^21, "
                                     "1 <= n_tets < 2^29)");
    Mesh *m = new Mesh();
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&m->device);
    m->n_nodes = n_nodes;
    m->n_tets = n_tets;
    m->n_gp = 4 * n_tets;
    m->bin_scale = (opt && opt->bin_scale > 0) ? opt->bin_scale : 0.5;
    m->max_steps = (opt && opt->max_steps > 0) ? opt->max_steps
                                               : (int)(8.0 * cbrt((double)n_tets)) + 64;
    m->profile = opt && opt->profile;
    m->tc_tile_opt = opt ? opt->tc_tile : 0;
    m->chol_tc_opt = opt ? opt->chol_tc : 0;
    if (m->tc_tile_opt != 0 && m->tc_tile_opt != 128 && m->tc_tile_opt != 256) {
        delete m;
        return set_error(FEM3_E_ARG, "tc_tile must be 0, 128 or 256");
    }
    auto fail = [&](int code) {
        fem3_mesh_free(reinterpret_cast<fem3_mesh>(m));
        return code;
    };
    if (m->profile) {
        for (int k = 0; k < 16; k++) cudaEventCreate(&m->ev[k]);
        m->ev_made = true;
    }
    // keep freed pool memory cached so that repeated uploads make no CUDA driver allocation
    {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, m->device) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    }
    int st;
    stage_begin(m, 0);
    if ((st = dev_alloc_t(m, &m->err, ERR_COUNT)) != FEM3_OK) return fail(st);
    if ((st = dev_alloc_t(m, &m->norms, 128)) != FEM3_OK) return fail(st);
    if (!(m->h_norms = pinned_block())) return fail(set_error(FEM3_E_OOM, "cudaMallocHost"));
    if (cudaMemsetAsync(m->err, 0, sizeof(int32_t) * ERR_COUNT, m->stream) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
    if ((st = dev_alloc_t(m, &m->verts, 3 * n_nodes)) != FEM3_OK) return fail(st);
    if ((st = dev_alloc_t(m, &m->tets, 4 * n_tets)) != FEM3_OK) return fail(st);
    cudaMemcpyKind kv = is_device_ptr(verts) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyKind kt = is_device_ptr(tets) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(m->verts, verts, sizeof(double) * 3 * n_nodes, kv, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->tets, tets, sizeof(int32_t) * 4 * n_tets, kt, m->stream) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "cudaMemcpyAsync"));
    if ((st = mesh_build(m, m->verts, m->tets)) != FEM3_OK) return fail(st);
    stage_end(m, 0);
    stage_begin(m, 1);
    if ((st = bins_build(m)) != FEM3_OK) return fail(st);
    stage_end(m, 1);
    const int64_t n = std::max<int64_t>(1, m->n_dof);
    if ((st = dev_alloc_t(m, &m->flags, 2 * ((n + 63) / 64) + 2)) != FEM3_OK) return fail(st);
    if ((st = dev_alloc(m, &m->solve_ws, sizeof(double) * 64 * 24 * ((n + 63) / 64))) != FEM3_OK)
        return fail(st);
    if ((st = dev_alloc(m, &m->solve_G, sizeof(double) * 2 * 3 * 64 * 64 * ((n + 63) / 64))) != FEM3_OK)
        return fail(st);
    if ((st = dev_alloc(m, &m->dinv, sizeof(double) * 64 * 64 * ((n + 63) / 64))) != FEM3_OK)
        return fail(st);
    {
        const int64_t nblk = (n + 63) / 64;
        if ((st = dev_alloc_t(m, &m->chol_flags, nblk * (nblk + 1) + 2)) != FEM3_OK)
            return fail(st);
    }
    if (cudaMemsetAsync(m->flags, 0, sizeof(int32_t) * (2 * ((n + 63) / 64) + 2), m->stream) != cudaSuccess)
        return fail(cuda_error(cudaGetLastError(), "cudaMemsetAsync"));
    for (int k = 0; k < 6; k++)
        if ((st = dev_alloc_t(m, &m->vec64[k], std::max<int64_t>(std::max<int64_t>(n, m->n_nodes),
                                                                 64 * 64))) != FEM3_OK)
            return fail(st);
    for (int k = 0; k < 2; k++)
        if ((st = dev_alloc_t(m, &m->vec32[k], n)) != FEM3_OK) return fail(st);
    if ((st = check_errors(m)) != FEM3_OK) return fail(st);
    *out = reinterpret_cast<fem3_mesh>(m);
    return FEM3_OK;
}

int fem3_mesh_info(fem3_mesh h, int64_t *n_dof, int64_t *n_gp, int32_t *dof_of_node) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m) return set_error(FEM3_E_ARG, "null mesh");
    if (n_dof) *n_dof = m->n_dof;
    if (n_gp) *n_gp = m->n_gp;
    if (dof_of_node) {
        FEM3_CUDA(cudaMemcpyAsync(dof_of_node, m->dof, sizeof(int32_t) * m->n_nodes,
                                  cudaMemcpyDeviceToHost, m->stream));
        FEM3_CUDA(cudaStreamSynchronize(m->stream));
    }
    return FEM3_OK;
}

int fem3_assemble(fem3_mesh h, const double alpha[3], const double K[3], int precision,
                  double *A_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !alpha || !K) return set_error(FEM3_E_ARG, "null argument");
    if (precision != FEM3_FP64 && precision != FEM3_TF32X3 && precision != FEM3_FP32 &&
        precision != FEM3_BF16X3)
        return set_error(FEM3_E_ARG, "unknown precision");
    for (int a = 0; a < 3; a++) {
        if (!(alpha[a] > 1.0 && alpha[a] <= 2.0))
            return set_error(FEM3_E_ARG, "alpha must lie in (1, 2]");
        if (!(K[a] > 0.0)) return set_error(FEM3_E_ARG, "K must be positive");
    }
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = m->n_dof;
    if (precision == FEM3_FP64 && !m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, n * n));
    if (precision != FEM3_FP64 && !m->A32) FEM3_TRY(dev_alloc_t(m, &m->A32, n * n));
    for (int a = 0; a < 3; a++) {
        m->alpha[a] = alpha[a];
        m->K[a] = K[a];
        m->s[a] = 1.0 / (2.0 * cos(M_PI * alpha[a] / 2.0));
        m->sK[a] = m->s[a] * K[a];
    }
    m->precision = precision;
    m->factored = false;
    m->ap_ready = false;
    m->integer_order = false;
    m->nonsym = false;
    kc_reset(m);
    FEM3_TRY(walk_tables(m, alpha));
    stage_begin(m, 3);
    if (precision == FEM3_TF32X3 || precision == FEM3_BF16X3)
        FEM3_TRY(contract_tc(m, precision == FEM3_BF16X3));
    else
        FEM3_TRY(contract(m, precision));
    stage_end(m, 3);
    if (A_out) {
        if (precision == FEM3_FP64) {
            FEM3_CUDA(cudaMemcpyAsync(A_out, m->A64, sizeof(double) * n * n,
                                      cudaMemcpyDeviceToDevice, m->stream));
        } else {
            FEM3_TRY(f32_to_f64(m->A32, A_out, n * n, m->stream));
            note_launch(m);
            if (precision == FEM3_TF32X3 || precision == FEM3_BF16X3) {
                // the tensor-core paths fill the lower triangle
                FEM3_TRY(sym_from_lower(A_out, n, m->stream));
                note_launch(m);
            }
        }
    }
    return FEM3_OK;
}

int fem3_assemble_part(fem3_mesh h, const double alpha[3], const double K[3], int precision,
                       int part, int nparts, double *A_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !A_out) return set_error(FEM3_E_ARG, "null argument");
    if (nparts < 1 || part < 0 || part >= nparts)
        return set_error(FEM3_E_ARG, "0 <= part < nparts required");
    m->part = part;
    m->nparts = nparts;
    const int st = fem3_assemble(h, alpha, K, precision, A_out, stream);
    m->part = 0;
    m->nparts = 1;
    // a part of the matrix (and of the tables) is no operator to solve with
    m->precision = -1;
    m->factored = false;
    m->ap_ready = false;
    return st;
}

int fem3_assemble_integer(fem3_mesh h, const double K[3], double *A_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !K) return set_error(FEM3_E_ARG, "null argument");
    for (int a = 0; a < 3; a++)
        if (!(K[a] > 0.0)) return set_error(FEM3_E_ARG, "K must be positive");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = m->n_dof;
    for (int a = 0; a < 3; a++) {
        m->alpha[a] = 2.0;
        m->K[a] = K[a];
        m->s[a] = -0.5;
        m->sK[a] = -0.5 * K[a];
    }
    m->precision = FEM3_FP64;
    m->factored = false;
    m->ap_ready = false;
    m->integer_order = true;
    m->nonsym = false;
    kc_reset(m);
    stage_begin(m, 3);
    FEM3_TRY(assemble_integer(m, K));
    stage_end(m, 3);
    if (A_out)
        FEM3_CUDA(cudaMemcpyAsync(A_out, m->A64, sizeof(double) * n * n, cudaMemcpyDeviceToDevice,
                                  m->stream));
    return FEM3_OK;
}

int fem3_assemble_form(fem3_mesh h, int axis, double alpha, double beta, int trial_left,
                       const double *c, int precision, double *K_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !K_out) return set_error(FEM3_E_ARG, "null argument");
    if (axis < 0 || axis > 2) return set_error(FEM3_E_ARG, "axis must be 0, 1 or 2");
    if (!(alpha >= 0.0 && alpha <= 1.0) || !(beta >= 0.0 && beta <= 1.0))
        return set_error(FEM3_E_ARG, "the orders of the general form lie in [0, 1]");
    if (precision != FEM3_FP64 && precision != FEM3_TF32X3 && precision != FEM3_FP32 &&
        precision != FEM3_BF16X3)
        return set_error(FEM3_E_ARG, "unknown precision");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = m->n_dof;
    // the tables of this axis are rewritten: no assembled operator remains for fem3_solve
    m->precision = -1;
    m->factored = false;
    m->ap_ready = false;
    m->integer_order = false;
    m->nonsym = false;
    kc_reset(m);
    if (precision == FEM3_FP64 && !m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, n * n));
    if (precision != FEM3_FP64 && !m->A32) FEM3_TRY(dev_alloc_t(m, &m->A32, n * n));
    if (!m->form_wc) FEM3_TRY(dev_alloc_t(m, &m->form_wc, 2 * m->n_gp));
    const void *cd = nullptr;
    void *owned = nullptr;
    if (c) FEM3_TRY(to_device(m, c, sizeof(double) * m->n_gp, &cd, &owned));
    // trial_left: D^a (trial) is the left operator and D^^b (test) the right one
    const double order_left = trial_left ? alpha : beta, order_right = trial_left ? beta : alpha;
    const bool test_right = trial_left != 0;
    int st = walk_tables_form(m, axis, order_left, order_right);
    if (st == FEM3_OK) st = weight_coef(m, (const double *)cd, m->form_wc);
    stage_begin(m, 3);
    if (st == FEM3_OK) {
        if (precision == FEM3_TF32X3 || precision == FEM3_BF16X3)
            st = contract_tc_form(m, axis, test_right, m->form_wc, precision == FEM3_BF16X3);
        else
            st = contract_form(m, axis, test_right, m->form_wc, precision);
    }
    stage_end(m, 3);
    if (st == FEM3_OK) {
        if (precision == FEM3_FP64) {
            cudaError_t e = cudaMemcpyAsync(K_out, m->A64, sizeof(double) * n * n,
                                            cudaMemcpyDeviceToDevice, m->stream);
            if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync");
        } else {
            st = f32_to_f64(m->A32, K_out, n * n, m->stream);
            note_launch(m);
        }
    }
    if (owned) cudaFreeAsync(owned, m->stream);
    return st;
}

int fem3_assemble_divergence(fem3_mesh h, const double beta[3], const double *p,
                             const double *q, int precision, double *A_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !beta || !p || !q) return set_error(FEM3_E_ARG, "null argument");
    for (int a = 0; a < 3; a++)
        if (!(beta[a] >= 0.0 && beta[a] <= 1.0))
            return set_error(FEM3_E_ARG, "beta must lie in [0, 1]");
    if (precision != FEM3_FP64 && precision != FEM3_TF32X3 && precision != FEM3_FP32 &&
        precision != FEM3_BF16X3)
        return set_error(FEM3_E_ARG, "unknown precision");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = m->n_dof;
    m->precision = -1;
    m->factored = false;
    m->ap_ready = false;
    m->integer_order = false;
    m->nonsym = false;
    kc_reset(m);
    const void *pd = nullptr, *qd = nullptr;
    void *po = nullptr, *qo = nullptr;
    FEM3_TRY(to_device(m, p, sizeof(double) * 3 * m->n_gp, &pd, &po));
    int st = to_device(m, q, sizeof(double) * 3 * m->n_gp, &qd, &qo);
    stage_begin(m, 3);
    if (st == FEM3_OK)
        st = assemble_divergence(m, beta, (const double *)pd, (const double *)qd, precision);
    stage_end(m, 3);
    if (st == FEM3_OK && A_out) {
        cudaError_t e = cudaMemcpyAsync(A_out, m->A_ns, sizeof(double) * n * n,
                                        cudaMemcpyDeviceToDevice, m->stream);
        if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync");
    }
    if (po) cudaFreeAsync(po, m->stream);
    if (qo) cudaFreeAsync(qo, m->stream);
    if (st == FEM3_OK) {
        m->precision = precision;
        m->nonsym = true;
    }
    return st;
}

int fem3_load(fem3_mesh h, const double *f, int nrhs, double *b, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !f || !b || nrhs < 1) return set_error(FEM3_E_ARG, "bad argument");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const void *fd = nullptr;
    void *owned = nullptr;
    FEM3_TRY(to_device(m, f, sizeof(double) * m->n_nodes * nrhs, &fd, &owned));
    int st = load_vector(m, (const double *)fd, nrhs, b);
    if (owned) cudaFreeAsync(owned, m->stream);
    return st;
}

int fem3_solve(fem3_mesh h, const double *f, int nrhs, double tol, int max_iter, double *u,
               int *iters_out, double *resid_out, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !f || !u || nrhs < 1) return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0) return set_error(FEM3_E_STATE, "solve before assemble");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = m->n_dof;
    if (n == 0) {
        if (iters_out) *iters_out = 0;
        if (resid_out) *resid_out = 0;
        return check_errors(m);
    }
    const void *fd = nullptr;
    void *owned = nullptr;
    FEM3_TRY(to_device(m, f, sizeof(double) * m->n_nodes * nrhs, &fd, &owned));
    double *b = nullptr;
    int st = FEM3_OK;
    cudaError_t e = cudaMallocAsync((void **)&b, sizeof(double) * std::max<int64_t>(1, n * nrhs), m->stream);
    if (e != cudaSuccess) st = cuda_error(e, "cudaMallocAsync");
    stage_begin(m, 4);
    if (st == FEM3_OK) st = load_vector(m, (const double *)fd, nrhs, b);
    stage_end(m, 4);
    if (m->nonsym) {
        // divergence form: GMRES per column, preconditioned by the SPD part's factor
        if (st == FEM3_OK && !m->factored) {
            stage_begin(m, 5);
            st = factor_nonsym(m);
            stage_end(m, 5);
            if (st == FEM3_OK) st = check_errors(m);
            if (st == FEM3_OK) m->factored = true;
        }
        stage_begin(m, 6);
        int it_max = 0;
        double worst = 0;
        for (int r = 0; r < nrhs && st == FEM3_OK; r++) {
            int it = 0;
            double rel = 0;
            st = gmres_solve(m, b + r * n, u + r * n, tol, max_iter > 0 ? max_iter : 300, &it, &rel);
            it_max = std::max(it_max, it);
            worst = std::max(worst, rel);
        }
        stage_end(m, 6);
        if (iters_out) *iters_out = it_max;
        if (resid_out) *resid_out = worst;
        if (b) cudaFreeAsync(b, m->stream);
        if (owned) cudaFreeAsync(owned, m->stream);
        int st2 = check_errors(m);
        stage_collect(m);
        return st != FEM3_OK ? st : st2;
    }
    if (st == FEM3_OK && !m->factored) {
        stage_begin(m, 5);
        st = factor(m);
        stage_end(m, 5);
        if (st == FEM3_OK) st = check_errors(m);
        if (st == FEM3_OK) m->factored = true;
    }
    stage_begin(m, 6);
    if (st == FEM3_OK) {
        if (m->precision == FEM3_FP64) {
            st = solve_direct(m, b, nrhs, u);
            if (st == FEM3_OK && resid_out) {
                double worst = 0;
                for (int r = 0; r < nrhs && st == FEM3_OK; r++) {
                    st = m->integer_order ? apply_integer(m, u + r * n, m->vec64[0])
                                          : apply_A64(m, u + r * n, m->vec64[0]);
                    double rel = 0;
                    if (st == FEM3_OK) st = residual_norm(m, b + r * n, m->vec64[0], &rel);
                    worst = std::max(worst, rel);
                }
                *resid_out = worst;
            }
            if (iters_out) *iters_out = 0;
        } else {
            st = solve_refined(m, b, nrhs, tol, max_iter > 0 ? max_iter : 50, u, iters_out, resid_out);
        }
    }
    stage_end(m, 6);
    if (b) cudaFreeAsync(b, m->stream);
    if (owned) cudaFreeAsync(owned, m->stream);
    int st2 = check_errors(m);
    stage_collect(m);
    return st != FEM3_OK ? st : st2;
}

// lambda = A^{-1} g, dK_i = -lambda^T (dA/dK_i) u, df = M^T lambda (g in m->vec64[2])
static int vjp_from_seed(Mesh *m, const double *u, const double *g, double tol, int max_iter,
                         double *dK, double *df) {
    double *lam = m->vec64[3];
    if (m->precision == FEM3_FP64) {
        FEM3_TRY(solve_direct(m, g, 1, lam));
    } else {
        FEM3_TRY(solve_refined(m, g, 1, tol, max_iter > 0 ? max_iter : 50, lam, nullptr, nullptr));
    }
    double forms[3];
    if (m->integer_order)
        FEM3_TRY(axis_forms_integer(m, u, lam, forms));
    else
        FEM3_TRY(axis_forms(m, u, lam, forms));
    for (int a = 0; a < 3; a++) dK[a] = -forms[a];
    if (df) FEM3_TRY(load_vector_T(m, lam, df));
    return check_errors(m);
}

int fem3_adjoint(fem3_mesh h, const double *u, const double *u_obs, double tol, int max_iter,
                 double *dJ_dK, double *dJ_df, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !u || !u_obs || !dJ_dK) return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0 || !m->factored) return set_error(FEM3_E_STATE, "adjoint before solve");
    if (m->nonsym) return set_error(FEM3_E_STATE, "no adjoint for the divergence form");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    double *res = m->vec64[2];
    FEM3_TRY(sub_vec(u, u_obs, res, m->n_dof, m->stream));
    note_launch(m);
    return vjp_from_seed(m, u, res, tol, max_iter, dJ_dK, dJ_df);
}

int fem3_vjp(fem3_mesh h, const double *u, const double *g, double tol, int max_iter,
             double *dK, double *df, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !u || !g || !dK) return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0 || !m->factored) return set_error(FEM3_E_STATE, "vjp before solve");
    if (m->nonsym) return set_error(FEM3_E_STATE, "no adjoint for the divergence form");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    double *seed = m->vec64[2];
    FEM3_CUDA(cudaMemcpyAsync(seed, g, sizeof(double) * m->n_dof, cudaMemcpyDeviceToDevice,
                              m->stream));
    return vjp_from_seed(m, u, seed, tol, max_iter, dK, df);
}

int fem3_paths(fem3_mesh h, int axis, int dir, const int64_t *gps, int64_t n_lines, int cap,
               int32_t *tet_out, double *r_in_out, double *r_out_out, int32_t *nseg_out,
               void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !gps || !tet_out || !r_in_out || !r_out_out || !nseg_out || cap < 1 ||
        axis < 0 || axis > 2 || (dir != 1 && dir != -1) || n_lines < 0)
        return set_error(FEM3_E_ARG, "bad argument");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    if (n_lines == 0) return FEM3_OK;
    return walk_paths(m, axis, dir, gps, n_lines, cap, tet_out, r_in_out, r_out_out, nseg_out);
}

int fem3_table_rows(fem3_mesh h, int axis, int dir, const int64_t *gps, int64_t n,
                    double *rows, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !gps || !rows || axis < 0 || axis > 2 || (dir != 1 && dir != -1) || n < 0)
        return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0) return set_error(FEM3_E_STATE, "tables before assemble");
    if (m->integer_order)
        return set_error(FEM3_E_STATE, "the integer-order assembly builds no derivative tables");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    return table_rows(m, axis, dir, gps, n, rows);
}

int fem3_sync(fem3_mesh h, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m) return set_error(FEM3_E_ARG, "null mesh");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    int st = check_errors(m);
    stage_collect(m);
    if (st == FEM3_OK) {
        unsigned long long segs = 0;
        FEM3_CUDA(cudaMemcpy(&segs, m->norms + kSegCounterSlot, sizeof(segs), cudaMemcpyDeviceToHost));
        m->segments = (int64_t)segs;
    }
    return st;
}

int fem3_stage_ms(fem3_mesh h, int stage, float *ms) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !ms || stage < 0 || stage > 6) return set_error(FEM3_E_ARG, "bad argument");
    *ms = m->stage_ms[stage];
    return FEM3_OK;
}

int fem3_tc_tile(fem3_mesh h, int32_t *tile_n, int32_t *tuned) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m) return set_error(FEM3_E_ARG, "null mesh");
    if (tile_n) *tile_n = m->tc_tile_used;
    if (tuned) *tuned = m->tc_tuned ? 1 : 0;
    return FEM3_OK;
}

int fem3_apply_lists(fem3_mesh h, int32_t *lists) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !lists) return set_error(FEM3_E_ARG, "bad argument");
    *lists = apply_lists_fit(m) ? 1 : 0;
    return FEM3_OK;
}

int fem3_contract_work(fem3_mesh h, double *flops, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !flops) return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0 || m->integer_order)
        return set_error(FEM3_E_STATE, "contraction work needs the tables of a fractional assemble");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    return contract_work(m, flops, nullptr);
}

int fem3_table_nnz(fem3_mesh h, int64_t *nnz, void *stream) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || !nnz) return set_error(FEM3_E_ARG, "bad argument");
    if (m->precision < 0 || m->integer_order)
        return set_error(FEM3_E_STATE, "table nonzeros need the tables of a fractional assemble");
    m->stream = reinterpret_cast<cudaStream_t>(stream);
    return contract_work(m, nullptr, nnz);
}

int fem3_kernel_ms(fem3_mesh h, int kclass, float *ms, int32_t *launches) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || kclass < 0 || kclass >= KC_COUNT) return set_error(FEM3_E_ARG, "bad argument");
    if (ms) *ms = m->kc_ms[kclass];
    if (launches) *launches = m->kc_n[kclass];
    return FEM3_OK;
}

int fem3_bin_stats(fem3_mesh h, int axis, int64_t *n_bins, int64_t *n_tmpl, int32_t *max_dof,
                   int32_t *max_gp) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m || axis < 0 || axis > 2) return set_error(FEM3_E_ARG, "bad argument");
    const AxisBins &B = m->bins[axis];
    if (n_bins) *n_bins = B.n_bins;
    if (n_tmpl) *n_tmpl = B.n_tmpl;
    if (max_dof) *max_dof = B.max_dof;
    if (max_gp) *max_gp = B.max_gp;
    return FEM3_OK;
}

int fem3_counters(fem3_mesh h, int64_t *segments, double *contract_flops, int64_t *table_bytes,
                  int64_t *launches) {
    Mesh *m = reinterpret_cast<Mesh *>(h);
    if (!m) return set_error(FEM3_E_ARG, "null mesh");
    if (launches) *launches = m->launches;
    if (segments) *segments = m->segments;
    if (contract_flops) *contract_flops = m->contract_flops;
    if (table_bytes) {
        int64_t t = 0;
        for (int a = 0; a < 3; a++) t += 2 * m->bins[a].tab_elems * (int64_t)sizeof(double);
        *table_bytes = t;
    }
    return FEM3_OK;
}

}  // extern "C"
