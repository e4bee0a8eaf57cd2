// Contraction A = sum_i s_i K_i (L_i^T W R_i + R_i^T W L_i) on CUDA cores, bin by bin
// (Section 2.1 element sum, Section 2.3 template: only dofs of a bin's template set can
// meet the bin's Gauss points, so each bin contributes a dense D_b x D_b block).
//
// Work item (bin, t1, t2), t1 <= t2, covers the 64 x 64 output tile of local dofs
// [64 t1, 64 t1 + 64) x [64 t2, 64 t2 + 64):
//   out(c1, c2) = sum_r w_r (L[c1][r] R[c2][r] + R[c1][r] L[c2][r])   (symmetric)
// and adds s K out(c1, c2) to A[dof c1][dof c2] (and to the mirror element when t1 < t2).
// TA is the arithmetic type (double for the FP64 form, float for the FP32 form).
#include <algorithm>
#include <cstring>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

constexpr int kTile = 64, kKC = 16;

// table entry (hi + lo pair) in the arithmetic type of the contraction
template <class TA>
__device__ __forceinline__ TA tab_value(const float2 *p) {
    const float2 v = *p;
    if constexpr (sizeof(TA) == 8) return (double)v.x + (double)v.y;
    else return v.x + v.y;
}

template <class TA>
__global__ void __launch_bounds__(256) k_contract_simt(
    const float2 *__restrict__ tabL, const float2 *__restrict__ tabR,
    const int4 *__restrict__ work, const int32_t *__restrict__ gp_off,
    const int32_t *__restrict__ gp_idx, const int32_t *__restrict__ dof_off,
    const int32_t *__restrict__ dof_idx, const int64_t *__restrict__ tab_off,
    const int32_t *__restrict__ tab_ld, const double *__restrict__ gw, double sK, TA *A,
    int64_t n_dof) {
    __shared__ TA sLa[kKC][kTile], sRa[kKC][kTile], sLb[kKC][kTile], sRb[kKC][kTile];
    __shared__ TA sw[kKC];
    const int4 wk = work[blockIdx.x];
    const int bin = wk.x, t1 = wk.y, t2 = wk.z;
    const int D = dof_off[bin + 1] - dof_off[bin];
    const int G = gp_off[bin + 1] - gp_off[bin];
    const int ld = tab_ld[bin];
    const float2 *L = tabL + tab_off[bin], *R = tabR + tab_off[bin];
    const int32_t *slots = gp_idx + gp_off[bin];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = t1 * kTile, b0 = t2 * kTile;

    TA acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = TA(0);

    for (int r0 = 0; r0 < G; r0 += kKC) {
        if (threadIdx.x < kKC) {
            int r = r0 + threadIdx.x;
            sw[threadIdx.x] = r < G ? TA(gw[slots[r]]) : TA(0);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int e = threadIdx.x + 256 * q;  // 0..1023 over 64 rows x 16 columns
            int c = e >> 4, k = e & 15, r = r0 + k;
            bool okr = r < G;
            int ca = a0 + c, cb = b0 + c;
            sLa[k][c] = (okr && ca < D) ? tab_value<TA>(L + (int64_t)ca * ld + r) : TA(0);
            sRa[k][c] = (okr && ca < D) ? tab_value<TA>(R + (int64_t)ca * ld + r) : TA(0);
            sLb[k][c] = (okr && cb < D) ? tab_value<TA>(L + (int64_t)cb * ld + r) : TA(0);
            sRb[k][c] = (okr && cb < D) ? tab_value<TA>(R + (int64_t)cb * ld + r) : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKC; k++) {
            TA la[4], ra[4], lb[4], rb[4];
            TA w = sw[k];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                la[i] = sLa[k][ty * 4 + i];
                ra[i] = sRa[k][ty * 4 + i];
                lb[i] = sLb[k][tx * 4 + i] * w;
                rb[i] = sRb[k][tx * 4 + i] * w;
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(la[i], rb[j], fma(ra[i], lb[j], acc[i][j]));
        }
        __syncthreads();
    }
    const int32_t *dofs = dof_idx + dof_off[bin];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int c1 = a0 + ty * 4 + i;
        if (c1 >= D) continue;
        int64_t j1 = dofs[c1];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int c2 = b0 + tx * 4 + j;
            if (c2 >= D) continue;
            int64_t j2 = dofs[c2];
            TA v = TA(sK) * acc[i][j];
            atomicAdd(&A[j1 * n_dof + j2], v);
            if (t1 != t2) atomicAdd(&A[j2 * n_dof + j1], v);
        }
    }
}

// Algorithmic work of the contraction (the sparse outer products the element sum needs):
// per bin (one CTA) and Gauss point column k, the nonzeros of L[.][k] and R[.][k] over the
// bin's template rows; adds 2 * 2 nnz(L) nnz(R) (two products, one multiply-add each) per
// Gauss point to *flops.
__global__ void __launch_bounds__(128) k_contract_work(
    const float2 *__restrict__ tabL, const float2 *__restrict__ tabR,
    const int32_t *__restrict__ gp_off, const int32_t *__restrict__ dof_off,
    const int64_t *__restrict__ tab_off, const int32_t *__restrict__ tab_ld, double *flops,
    unsigned long long *nnz) {
    const int b = blockIdx.x;
    const int D = dof_off[b + 1] - dof_off[b];
    const int G = gp_off[b + 1] - gp_off[b];
    const int ld = tab_ld[b];
    const float2 *L = tabL + tab_off[b], *R = tabR + tab_off[b];
    double acc = 0.0;
    unsigned long long cnt = 0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        int nl = 0, nr = 0;
        for (int c = 0; c < D; c++) {
            const float2 a = L[(int64_t)c * ld + k], r = R[(int64_t)c * ld + k];
            nl += (a.x != 0.f || a.y != 0.f);
            nr += (r.x != 0.f || r.y != 0.f);
        }
        acc += 4.0 * (double)nl * (double)nr;
        cnt += (unsigned long long)(nl + nr);
    }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(flops, acc);
    if ((threadIdx.x & 31) == 0 && cnt != 0) atomicAdd(nnz, cnt);
}

// One product of the general form (c D^a u, D^^b v), all 64 x 64 tile pairs of each bin:
// out(c1, c2) = sum_r wc_r T[c1][r] S[c2][r] (T the test side's table, S the trial side's,
// wc the Gauss weight times the coefficient) added to K[dof c1][dof c2].
template <class TA>
__global__ void __launch_bounds__(256) k_contract_form(
    const float2 *__restrict__ tabT, const float2 *__restrict__ tabS,
    const int4 *__restrict__ work, const int32_t *__restrict__ gp_off,
    const int32_t *__restrict__ gp_idx, const int32_t *__restrict__ dof_off,
    const int32_t *__restrict__ dof_idx, const int64_t *__restrict__ tab_off,
    const int32_t *__restrict__ tab_ld, const double *__restrict__ wc, TA *K, int64_t n_dof) {
    __shared__ TA sT[kKC][kTile], sS[kKC][kTile];
    __shared__ TA sw[kKC];
    const int4 wk = work[blockIdx.x];
    const int bin = wk.x, t1 = wk.y, t2 = wk.z;
    const int D = dof_off[bin + 1] - dof_off[bin];
    const int G = gp_off[bin + 1] - gp_off[bin];
    const int ld = tab_ld[bin];
    const float2 *T = tabT + tab_off[bin], *S = tabS + tab_off[bin];
    const int32_t *slots = gp_idx + gp_off[bin];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int a0 = t1 * kTile, b0 = t2 * kTile;
    TA acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = TA(0);
    for (int r0 = 0; r0 < G; r0 += kKC) {
        if (threadIdx.x < kKC) {
            const int r = r0 + threadIdx.x;
            sw[threadIdx.x] = r < G ? TA(wc[slots[r]]) : TA(0);
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int e = threadIdx.x + 256 * q;
            const int c = e >> 4, k = e & 15, r = r0 + k;
            const bool okr = r < G;
            const int ca = a0 + c, cb = b0 + c;
            sT[k][c] = (okr && ca < D) ? tab_value<TA>(T + (int64_t)ca * ld + r) : TA(0);
            sS[k][c] = (okr && cb < D) ? tab_value<TA>(S + (int64_t)cb * ld + r) : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kKC; k++) {
            TA ta[4], sb[4];
            const TA w = sw[k];
#pragma unroll
            for (int i = 0; i < 4; i++) {
                ta[i] = sT[k][ty * 4 + i];
                sb[i] = sS[k][tx * 4 + i] * w;
            }
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(ta[i], sb[j], acc[i][j]);
        }
        __syncthreads();
    }
    const int32_t *dofs = dof_idx + dof_off[bin];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int c1 = a0 + ty * 4 + i;
        if (c1 >= D) continue;
        const int64_t j1 = dofs[c1];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int c2 = b0 + tx * 4 + j;
            if (c2 >= D) continue;
            atomicAdd(&K[j1 * n_dof + dofs[c2]], acc[i][j]);
        }
    }
}

// wc[g] = w[g] c[g] (c NULL: w)
__global__ void k_weight_coef(const double *__restrict__ w, const double *__restrict__ c,
                              int64_t n, double *wc) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < n) wc[g] = c ? w[g] * c[g] : w[g];
}

}  // namespace

int weight_coef(Mesh *m, const double *c_gp, double *wc_gp) {
    k_weight_coef<<<(unsigned)((m->n_gp + 255) / 256), 256, 0, m->stream>>>(m->gw, c_gp, m->n_gp,
                                                                             wc_gp);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// K = T^T diag(wc) S over one axis's bins on CUDA cores (FP64 into A64 or FP32 into A32),
// T the test side's table (R if test_right), S the trial side's
int contract_form(Mesh *m, int axis, bool test_right, const double *wc_gp, int precision) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    AxisBins &B = m->bins[axis];
    if (!B.form_work) {
        std::vector<int4> work;
        for (int b = 0; b < B.n_bins; b++) {
            const int D = B.h_dof_off[b + 1] - B.h_dof_off[b];
            const int G = B.h_gp_off[b + 1] - B.h_gp_off[b];
            if (D == 0 || G == 0) continue;
            const int nt = (D + kTile - 1) / kTile;
            for (int t1 = 0; t1 < nt; t1++)
                for (int t2 = 0; t2 < nt; t2++) work.push_back(make_int4(b, t1, t2, 0));
        }
        B.n_form_work = (int)work.size();
        FEM3_TRY(dev_alloc_t(m, &B.form_work, std::max(1, B.n_form_work)));
        if (B.n_form_work)
            FEM3_CUDA(cudaMemcpyAsync(B.form_work, work.data(), sizeof(int4) * work.size(),
                                      cudaMemcpyHostToDevice, s));
        // the pageable source must outlive the copy
        FEM3_CUDA(cudaStreamSynchronize(s));
    }
    const float2 *T = test_right ? m->tabR[axis] : m->tabL[axis];
    const float2 *S = test_right ? m->tabL[axis] : m->tabR[axis];
    if (precision == FEM3_FP64) {
        FEM3_CUDA(cudaMemsetAsync(m->A64, 0, sizeof(double) * n * n, s));
    } else {
        FEM3_CUDA(cudaMemsetAsync(m->A32, 0, sizeof(float) * n * n, s));
    }
    if (B.n_form_work) {
        kc_begin(m, KC_CONTRACT);
        if (precision == FEM3_FP64)
            k_contract_form<double><<<B.n_form_work, 256, 0, s>>>(
                T, S, B.form_work, B.gp_off, B.gp_idx, B.dof_off, B.dof_idx, B.tab_off, B.tab_ld,
                wc_gp, m->A64, n);
        else
            k_contract_form<float><<<B.n_form_work, 256, 0, s>>>(
                T, S, B.form_work, B.gp_off, B.gp_idx, B.dof_off, B.dof_idx, B.tab_off, B.tab_ld,
                wc_gp, m->A32, n);
        kc_end(m, KC_CONTRACT);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int contract_work(Mesh *m, double *flops_out, int64_t *nnz_out) {
    cudaStream_t s = m->stream;
    double *d = m->norms + 121;
    unsigned long long *c = reinterpret_cast<unsigned long long *>(m->norms + 122);
    FEM3_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(double), s));
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        if (B.n_bins == 0 || B.n_tmpl == 0) continue;
        k_contract_work<<<B.n_bins, 128, 0, s>>>(m->tabL[axis], m->tabR[axis], B.gp_off,
                                                  B.dof_off, B.tab_off, B.tab_ld, d, c);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    FEM3_CUDA(cudaMemcpyAsync(m->h_norms + 121, d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    if (flops_out) *flops_out = m->h_norms[121];
    if (nnz_out) {
        unsigned long long v;
        memcpy(&v, m->h_norms + 122, sizeof(v));
        *nnz_out = (int64_t)v;
    }
    return FEM3_OK;
}

int contract(Mesh *m, int precision) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    double flops = 0;
    if (precision == FEM3_FP64) {
        FEM3_CUDA(cudaMemsetAsync(m->A64, 0, sizeof(double) * n * n, s));
    } else {
        FEM3_CUDA(cudaMemsetAsync(m->A32, 0, sizeof(float) * n * n, s));
    }
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        for (int b = 0; b < B.n_bins; b++) {
            double D = B.h_dof_off[b + 1] - B.h_dof_off[b];
            double G = B.h_gp_off[b + 1] - B.h_gp_off[b];
            flops += 2.0 * D * D * G;
        }
        if (!B.n_work) continue;
        // the work items of this part's bins (the list is in bin order)
        int b0, b1;
        part_bins(m, axis, b0, b1);
        const auto lb = [&](int b) {
            return (int)(std::lower_bound(B.h_work.begin(), B.h_work.end(), b,
                                          [](const int4 &x, int v) { return x.x < v; }) -
                         B.h_work.begin());
        };
        const int w0 = lb(b0), nw = lb(b1) - w0;
        if (nw <= 0) continue;
        kc_begin(m, KC_CONTRACT);
        if (precision == FEM3_FP64)
            k_contract_simt<double><<<nw, 256, 0, s>>>(
                m->tabL[axis], m->tabR[axis], B.work + w0, B.gp_off, B.gp_idx, B.dof_off,
                B.dof_idx, B.tab_off, B.tab_ld, m->gw, m->sK[axis], m->A64, n);
        else
            k_contract_simt<float><<<nw, 256, 0, s>>>(
                m->tabL[axis], m->tabR[axis], B.work + w0, B.gp_off, B.gp_idx, B.dof_off,
                B.dof_idx, B.tab_off, B.tab_ld, m->gw, m->sK[axis], m->A32, n);
        kc_end(m, KC_CONTRACT);
        note_launch(m);
    }
    m->contract_flops = flops;
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

}  // namespace fem3
