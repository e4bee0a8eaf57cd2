// Section 3's divergence-form operator (eq. "equ:sfde2") and its non-symmetric solve.
//
//   a(u, v) = -sum_i ((p_i D_L^{b_i} u, D_i v) - (q_i D_R^{b_i} u, D_i v)),  A[k][l] = a(psi_l, psi_k)
//
// With the one-sided order-1 derivatives D_L^1 v = dv/dx_i and D_R^1 v = -dv/dx_i, each axis
// contributes two terms of the general form of Section 2.1:
//   -(p D_L^b u, D_i v) = (p D_L^b u, D_R^1 v)   (trial left, order b; test right, order 1)
//    (q D_R^b u, D_i v) = (q D_R^b u, D_L^1 v)   (trial right, order b; test left, order 1)
// so the matrix is the sum of six fem3_assemble_form terms, accumulated in FP64.
//
// The solve: A is not symmetric; its symmetric part S = (A + A^T)/2 is negative definite for
// positive p_i, q_i (the form is minus an elliptic one), so M = -S is SPD and its FP64
// Cholesky factor (the tile-task factorisation) preconditions restarted GMRES on A: right
// preconditioning, classical Gram-Schmidt with one reorthogonalisation, Givens rotations
// on the host, the true residual b - A x checked at every restart.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

constexpr int kRestart = 30;

__global__ void k_add_f64(const double *__restrict__ x, int64_t n, double *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}
__global__ void k_add_f32(const float *__restrict__ x, int64_t n, double *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += (double)x[i];
}
// M = -(A + A^T) / 2
__global__ void k_neg_sym(const double *__restrict__ A, int64_t n, double *Mout) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e - i * n;
    Mout[e] = -0.5 * (A[i * n + j] + A[j * n + i]);
}
// y = A x (one warp per row)
__global__ void k_gemv(const double *__restrict__ A, const double *__restrict__ x, int64_t n,
                       double *y) {
    const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t c = lane; c < n; c += 32) acc = fma(A[row * n + c], x[c], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[row] = acc;
}
// h[j] = V_j . w for j < k (one block per j)
__global__ void k_multidot(const double *__restrict__ V, int64_t n, const double *__restrict__ w,
                           double *h) {
    __shared__ double red[8];
    const double *v = V + blockIdx.x * n;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) acc = fma(v[r], w[r], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
        h[blockIdx.x] = s;
    }
}
// w -= sum_{j<k} h[j] V_j
__global__ void k_multiaxpy(const double *__restrict__ V, int64_t n, int k,
                            const double *__restrict__ h, double *w) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double acc = 0.0;
    for (int j = 0; j < k; j++) acc = fma(h[j], V[j * n + r], acc);
    w[r] -= acc;
}
// y = sum_{j<k} c[j] V_j
__global__ void k_combine(const double *__restrict__ V, int64_t n, int k,
                          const double *__restrict__ c, double *y) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    double acc = 0.0;
    for (int j = 0; j < k; j++) acc = fma(c[j], V[j * n + r], acc);
    y[r] = acc;
}
__global__ void k_scale_to(const double *__restrict__ x, int64_t n, double a, double *y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i];
}
inline unsigned g256(int64_t n) { return (unsigned)(n > 0 ? (n + 255) / 256 : 1); }

}  // namespace

// Divergence-form matrix into m->A_ns (FP64), six general-form terms; precision as in
// fem3_assemble_form (the tables' products), the sum in FP64.
int assemble_divergence(Mesh *m, const double beta[3], const double *p_d, const double *q_d,
                        int precision) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof, ng = m->n_gp;
    if (!m->A_ns) FEM3_TRY(dev_alloc_t(m, &m->A_ns, std::max<int64_t>(1, n * n)));
    if (precision == FEM3_FP64 && !m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, n * n));
    if (precision != FEM3_FP64 && !m->A32) FEM3_TRY(dev_alloc_t(m, &m->A32, n * n));
    if (!m->form_wc) FEM3_TRY(dev_alloc_t(m, &m->form_wc, 2 * ng));
    FEM3_CUDA(cudaMemsetAsync(m->A_ns, 0, sizeof(double) * n * n, s));
    for (int axis = 0; axis < 3; axis++) {
        for (int term = 0; term < 2; term++) {
            // term 0: trial left (order b), test right (order 1), coefficient p
            // term 1: trial right (order b), test left (order 1), coefficient q
            const double oleft = term == 0 ? beta[axis] : 1.0;
            const double oright = term == 0 ? 1.0 : beta[axis];
            const double *c = (term == 0 ? p_d : q_d) + axis * ng;
            FEM3_TRY(walk_tables_form(m, axis, oleft, oright));
            FEM3_TRY(weight_coef(m, c, m->form_wc));
            const bool test_right = term == 0;
            if (precision == FEM3_TF32X3 || precision == FEM3_BF16X3)
                FEM3_TRY(contract_tc_form(m, axis, test_right, m->form_wc, precision == FEM3_BF16X3));
            else
                FEM3_TRY(contract_form(m, axis, test_right, m->form_wc, precision));
            if (precision == FEM3_FP64)
                k_add_f64<<<g256(n * n), 256, 0, s>>>(m->A64, n * n, m->A_ns);
            else
                k_add_f32<<<g256(n * n), 256, 0, s>>>(m->A32, n * n, m->A_ns);
            note_launch(m);
        }
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// Preconditioner: the FP64 Cholesky factor of M = -(A + A^T)/2 (in A64).
int factor_nonsym(Mesh *m) {
    const int64_t n = m->n_dof;
    if (!m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, n * n));
    k_neg_sym<<<g256(n * n), 256, 0, m->stream>>>(m->A_ns, n, m->A64);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    const int prec = m->precision;
    m->precision = FEM3_FP64;   // the FP64 tile-task factorisation of A64
    const int st = factor(m);
    m->precision = prec;
    return st;
}

// GMRES(30) on A x = b (A = m->A_ns), right-preconditioned by M^{-1} (M = -S: the system
// solved is (-A) x = -b, the same x); x starts at 0.  Stops when ||b - A x|| <= tol ||b||
// (true residual at a restart) or after max_iter Arnoldi steps.
int gmres_solve(Mesh *m, const double *b, double *x, double tol, int max_iter, int *iters,
                double *resid) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    const int mr = kRestart;
    double *V = nullptr, *w = nullptr, *z = nullptr, *bn = nullptr, *hd = nullptr;
    FEM3_CUDA(cudaMallocAsync((void **)&V, sizeof(double) * n * (mr + 1), s));
    FEM3_CUDA(cudaMallocAsync((void **)&w, sizeof(double) * n, s));
    FEM3_CUDA(cudaMallocAsync((void **)&z, sizeof(double) * n, s));
    FEM3_CUDA(cudaMallocAsync((void **)&bn, sizeof(double) * n, s));
    FEM3_CUDA(cudaMallocAsync((void **)&hd, sizeof(double) * (mr + 2), s));
    double *h_h = m->h_norms;   // pinned host mirror (>= 64 values)
    int st = FEM3_OK;
    auto sync_read = [&](const double *d, int cnt) -> int {
        FEM3_CUDA(cudaMemcpyAsync(h_h, d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s));
        FEM3_CUDA(cudaStreamSynchronize(s));
        return FEM3_OK;
    };
    auto norm = [&](const double *v, double *out) -> int {
        k_multidot<<<1, 256, 0, s>>>(v, n, v, hd);
        note_launch(m);
        FEM3_TRY(sync_read(hd, 1));
        *out = sqrt(std::max(0.0, h_h[0]));
        return FEM3_OK;
    };
    // (-A) x = -b: bn = -b
    k_scale_to<<<g256(n), 256, 0, s>>>(b, n, -1.0, bn);
    note_launch(m);
    FEM3_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    double bnorm = 0.0;
    if ((st = norm(bn, &bnorm)) != FEM3_OK) goto done;
    {
        int total = 0;
        double rel = 1.0;
        double beta = bnorm;
        // r0 = bn (x = 0)
        FEM3_CUDA(cudaMemcpyAsync(V, bn, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if (bnorm == 0.0) {
            rel = 0.0;
        }
        std::vector<double> H((mr + 1) * mr), cs(mr), sn(mr), g(mr + 1), y(mr);
        while (rel > tol && total < max_iter && st == FEM3_OK) {
            k_scale_to<<<g256(n), 256, 0, s>>>(V, n, 1.0 / beta, V);
            note_launch(m);
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            for (; k < mr && total < max_iter; k++, total++) {
                double *vk = V + (int64_t)k * n, *vn = V + (int64_t)(k + 1) * n;
                // w = (-A) M^{-1} v_k
                if ((st = solve_direct(m, vk, 1, z)) != FEM3_OK) break;
                k_gemv<<<g256(32 * n), 256, 0, s>>>(m->A_ns, z, n, w);
                note_launch(m);
                k_scale_to<<<g256(n), 256, 0, s>>>(w, n, -1.0, w);
                note_launch(m);
                // classical Gram-Schmidt, twice
                std::vector<double> hcol(k + 2, 0.0);
                for (int pass = 0; pass < 2; pass++) {
                    k_multidot<<<k + 1, 256, 0, s>>>(V, n, w, hd);
                    note_launch(m);
                    k_multiaxpy<<<g256(n), 256, 0, s>>>(V, n, k + 1, hd, w);
                    note_launch(m);
                    if ((st = sync_read(hd, k + 1)) != FEM3_OK) break;
                    for (int j = 0; j <= k; j++) hcol[j] += h_h[j];
                }
                if (st != FEM3_OK) break;
                double hn = 0.0;
                if ((st = norm(w, &hn)) != FEM3_OK) break;
                hcol[k + 1] = hn;
                if (hn > 0.0) {
                    k_scale_to<<<g256(n), 256, 0, s>>>(w, n, 1.0 / hn, vn);
                    note_launch(m);
                }
                // previous rotations, then a new one that zeroes hcol[k + 1]
                for (int j = 0; j < k; j++) {
                    const double t = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
                    hcol[j + 1] = -sn[j] * hcol[j] + cs[j] * hcol[j + 1];
                    hcol[j] = t;
                }
                const double den = hypot(hcol[k], hcol[k + 1]);
                cs[k] = den > 0 ? hcol[k] / den : 1.0;
                sn[k] = den > 0 ? hcol[k + 1] / den : 0.0;
                hcol[k] = den;
                hcol[k + 1] = 0.0;
                g[k + 1] = -sn[k] * g[k];
                g[k] = cs[k] * g[k];
                for (int j = 0; j <= k; j++) H[j * mr + k] = hcol[j];
                if (fabs(g[k + 1]) <= tol * bnorm * 0.1 || hn == 0.0) {
                    k++;
                    total++;
                    break;
                }
            }
            if (st != FEM3_OK) break;
            // y = H^{-1} g (upper triangular k x k), x += M^{-1} V y
            for (int i = k - 1; i >= 0; i--) {
                double t = g[i];
                for (int j = i + 1; j < k; j++) t -= H[i * mr + j] * y[j];
                y[i] = H[i * mr + i] != 0.0 ? t / H[i * mr + i] : 0.0;
            }
            for (int j = 0; j < k; j++) h_h[j] = y[j];
            FEM3_CUDA(cudaMemcpyAsync(hd, h_h, sizeof(double) * k, cudaMemcpyHostToDevice, s));
            k_combine<<<g256(n), 256, 0, s>>>(V, n, k, hd, w);
            note_launch(m);
            if ((st = solve_direct(m, w, 1, z)) != FEM3_OK) break;
            k_add_f64<<<g256(n), 256, 0, s>>>(z, n, x);
            note_launch(m);
            // true residual of (-A) x = bn: V_0 = bn - (-A x) = bn + A x
            k_gemv<<<g256(32 * n), 256, 0, s>>>(m->A_ns, x, n, w);
            note_launch(m);
            FEM3_CUDA(cudaMemcpyAsync(V, bn, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            k_add_f64<<<g256(n), 256, 0, s>>>(w, n, V);
            note_launch(m);
            if ((st = norm(V, &beta)) != FEM3_OK) break;
            rel = bnorm > 0 ? beta / bnorm : 0.0;
        }
        if (iters) *iters = total;
        if (resid) *resid = rel;
        if (st == FEM3_OK && !(rel <= tol))
            st = set_error(FEM3_E_NO_CONVERGE, "GMRES did not reach the tolerance");
    }
done:
    cudaFreeAsync(V, s);
    cudaFreeAsync(w, s);
    cudaFreeAsync(z, s);
    cudaFreeAsync(bn, s);
    cudaFreeAsync(hd, s);
    return st;
}

}  // namespace fem3
