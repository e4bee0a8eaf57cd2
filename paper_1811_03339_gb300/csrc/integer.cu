// Integer-order special case (alpha_i = 2 on every axis, Table 4's integer-order columns):
// the operator -sum_i K_i d^2 u / dx_i^2 has the local P1 stiffness matrix
//   A_jk = sum_i K_i sum_T |T| (d lambda_j / dx_i)|_T (d lambda_k / dx_i)|_T,
// so it is assembled tet by tet from the volume-coordinate gradients of the mesh records
// (no path walk, no tables).  The fractional assembly at alpha_i = 2 gives the same matrix
// (its one-sided order-1 derivatives are the slope on the Gauss point's tet, and
// s_i = -1/2); this is its fast special case.  The matrix is FP64 and is solved by the
// FP64 form.
#include "fem3_impl.cuh"

namespace fem3 {

namespace {

// one thread per tet: the 4 x 4 element matrix added into the dof rows and columns
__global__ void k_p1_stiffness(const double *__restrict__ M, const double *__restrict__ vol,
                               const int32_t *__restrict__ tets, const int32_t *__restrict__ dof,
                               int64_t n_tets, double K0, double K1, double K2, double *A,
                               int64_t n) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    const double *Mt = M + 16 * t;
    const double v = vol[t];
    int32_t j[4];
    double g[4][3];
    for (int a = 0; a < 4; a++) {
        j[a] = dof[tets[4 * t + a]];
        for (int i = 0; i < 3; i++) g[a][i] = Mt[4 * a + 1 + i];
    }
    for (int a = 0; a < 4; a++) {
        if (j[a] < 0) continue;
        for (int b = 0; b < 4; b++) {
            if (j[b] < 0) continue;
            const double e = v * (K0 * g[a][0] * g[b][0] + K1 * g[a][1] * g[b][1] +
                                  K2 * g[a][2] * g[b][2]);
            atomicAdd(&A[(int64_t)j[a] * n + j[b]], e);
        }
    }
}

// out[i] += sum_T |T| (d_i u_h)(d_i lambda_h) over the tets (u_h, lambda_h the P1
// functions of the dof vectors, zero on boundary vertices): lambda^T (dA/dK_i) u
__global__ void k_p1_axis_forms(const double *__restrict__ M, const double *__restrict__ vol,
                                const int32_t *__restrict__ tets,
                                const int32_t *__restrict__ dof, int64_t n_tets,
                                const double *__restrict__ u, const double *__restrict__ lam,
                                double *out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double f[3] = {0.0, 0.0, 0.0};
    if (t < n_tets) {
        const double *Mt = M + 16 * t;
        double du[3] = {0, 0, 0}, dl[3] = {0, 0, 0};
        for (int a = 0; a < 4; a++) {
            const int32_t j = dof[tets[4 * t + a]];
            if (j < 0) continue;
            for (int i = 0; i < 3; i++) {
                du[i] += Mt[4 * a + 1 + i] * u[j];
                dl[i] += Mt[4 * a + 1 + i] * lam[j];
            }
        }
        for (int i = 0; i < 3; i++) f[i] = vol[t] * du[i] * dl[i];
    }
    for (int i = 0; i < 3; i++) {
        double x = f[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x != 0.0) atomicAdd(&out[i], x);
    }
}

// y += A x tet by tet (the element matrices of k_p1_stiffness applied to x; the assembled
// matrix itself is overwritten by its factorisation)
__global__ void k_p1_apply(const double *__restrict__ M, const double *__restrict__ vol,
                           const int32_t *__restrict__ tets, const int32_t *__restrict__ dof,
                           int64_t n_tets, double K0, double K1, double K2,
                           const double *__restrict__ x, double *y) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    const double *Mt = M + 16 * t;
    int32_t j[4];
    double dx[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; a++) {
        j[a] = dof[tets[4 * t + a]];
        if (j[a] < 0) continue;
        for (int i = 0; i < 3; i++) dx[i] += Mt[4 * a + 1 + i] * x[j[a]];
    }
    const double v = vol[t];
    for (int a = 0; a < 4; a++) {
        if (j[a] < 0) continue;
        const double e = v * (K0 * Mt[4 * a + 1] * dx[0] + K1 * Mt[4 * a + 2] * dx[1] +
                              K2 * Mt[4 * a + 3] * dx[2]);
        atomicAdd(&y[j[a]], e);
    }
}

inline unsigned grid_tets(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int assemble_integer(Mesh *m, const double K[3]) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    if (!m->A64) FEM3_TRY(dev_alloc_t(m, &m->A64, n * n));
    FEM3_CUDA(cudaMemsetAsync(m->A64, 0, sizeof(double) * n * n, s));
    if (n > 0 && m->n_tets > 0) {
        kc_begin(m, KC_CONTRACT);
        k_p1_stiffness<<<grid_tets(m->n_tets), 256, 0, s>>>(m->M, m->vol, m->tets, m->dof,
                                                             m->n_tets, K[0], K[1], K[2], m->A64, n);
        kc_end(m, KC_CONTRACT);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int apply_integer(Mesh *m, const double *x, double *y) {
    FEM3_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * m->n_dof, m->stream));
    if (m->n_dof > 0 && m->n_tets > 0) {
        k_p1_apply<<<grid_tets(m->n_tets), 256, 0, m->stream>>>(
            m->M, m->vol, m->tets, m->dof, m->n_tets, m->K[0], m->K[1], m->K[2], x, y);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int axis_forms_integer(Mesh *m, const double *u, const double *lam, double out[3]) {
    cudaStream_t s = m->stream;
    FEM3_CUDA(cudaMemsetAsync(m->norms, 0, sizeof(double) * 3, s));
    if (m->n_tets > 0) {
        k_p1_axis_forms<<<grid_tets(m->n_tets), 256, 0, s>>>(m->M, m->vol, m->tets, m->dof,
                                                              m->n_tets, u, lam, m->norms);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    FEM3_CUDA(cudaMemcpyAsync(m->h_norms, m->norms, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; a++) out[a] = m->h_norms[a];
    return FEM3_OK;
}

}  // namespace fem3
