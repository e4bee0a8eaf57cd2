// Load vector, dense SPD solve and iterative refinement.
//
//  - b = M f with the P1 mass matrix (|T|/20 (1 + delta_ab) per tet), the weak
//    right-hand side (f, v) of Section 3.
//  - Right-looking blocked Cholesky A = L L^T (block 64): diagonal block in shared
//    memory, panel triangular solve, trailing symmetric update; row-major storage: the
//    tiles below the diagonal in A's lower triangle, each diagonal tile as its inverse
//    L_jj^{-1} (all the solves use).  TF is double (FP64 form) or float (mixed forms).
//  - Blocked forward / backward substitution.
//  - Refinement for the mixed forms: r = b - A u with A u applied in FP64 from the FP64
//    derivative tables (A u = sum_i s_i K_i (L_i^T W (R_i u) + R_i^T W (L_i u))), the
//    correction solved with the FP32 factor.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

__global__ void k_load(const int32_t *__restrict__ tets, const double *__restrict__ vol,
                       const int32_t *__restrict__ dof, int64_t n_tets, int64_t n_nodes,
                       int64_t n_dof, const double *__restrict__ f, int nrhs, double *b) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    int32_t v[4];
    for (int k = 0; k < 4; k++) v[k] = tets[4 * t + k];
    double c = vol[t] / 20.0;
    for (int r = 0; r < nrhs; r++) {
        const double *fr = f + (int64_t)r * n_nodes;
        double fv[4], fs = 0;
        for (int k = 0; k < 4; k++) { fv[k] = fr[v[k]]; fs += fv[k]; }
        for (int k = 0; k < 4; k++) {
            int32_t j = dof[v[k]];
            if (j >= 0) atomicAdd(&b[(int64_t)r * n_dof + j], c * (fs + fv[k]));
        }
    }
}

__global__ void k_load_T(const int32_t *__restrict__ tets, const double *__restrict__ vol,
                         const int32_t *__restrict__ dof, int64_t n_tets,
                         const double *__restrict__ lam, double *out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    int32_t v[4];
    double lv[4], ls = 0;
    for (int k = 0; k < 4; k++) {
        v[k] = tets[4 * t + k];
        int32_t j = dof[v[k]];
        lv[k] = j >= 0 ? lam[j] : 0.0;
        ls += lv[k];
    }
    double c = vol[t] / 20.0;
    for (int k = 0; k < 4; k++) atomicAdd(&out[v[k]], c * (ls + lv[k]));
}

#include "chol_smem.cuh"

// ---------------------------------------------------------------------------------
// Tile-task Cholesky in one launch.  CTA 0 runs the diagonal chain: for each block
// column j it applies the last update (k = j - 1) to the diagonal tile, factors it
// (L_jj and L_jj^{-1}), solves the tile below it, L_{j+1,j} = A_{j+1,j} L_jj^{-T}, and
// keeps that tile in shared memory for the next diagonal update, so the critical path
// never leaves one SM.  The other CTAs take tasks W(i, j) over the lower 64 x 64 tiles
// from an atomic ticket, column by column: W(i, j) subtracts L_ik L_jk^T for k < j (for a
// diagonal tile k < j - 1), each as soon as tiles (i, k) and (j, k) are final; the
// diagonal and sub-diagonal tiles are then stored for the chain ("updated" flag U),
// every other tile is solved with L_jj^{-1} once the chain has published it and stored
// as final (flag F).  Every task depends only on tiles of earlier columns (or, for the
// solve, on the chain's step j), and tickets are taken in column order, so the earliest
// unfinished claimed task always proceeds and the launch needs no co-residency.  Waits
// are bounded; a wait that expires sets the abort word, which every other wait also
// watches, and records ERR_CHOL.
// flags: F [0, ntask), U [ntask, 2 ntask), ticket [2 ntask], abort word [2 ntask + 1];
// all zero at launch.
// ---------------------------------------------------------------------------------
constexpr int kTileLd = NB + 4;
constexpr int kCholTilesSmem = 4 * NB * kTileLd;   // elements of dynamic shared memory

__device__ __forceinline__ int tile_id(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ bool wait_tile(const int *f, int *abort_w, int32_t *err) {
    int spins = 0;
    while (ld_acquire_gpu(f) == 0) {
        if (ld_acquire_gpu(abort_w) != 0) return false;
        if (++spins > kSpinLimit) {
            atomicAdd(&err[ERR_CHOL], 1);
            atomicExch(abort_w, 1);
            return false;
        }
        if (spins > 64) __nanosleep(128);   // 150 pollers on one L2 line slow its owner
    }
    return true;
}

// Tile loads, 512 threads: warp w reads rows 4w .. 4w + 3, lanes over the columns (each
// load instruction covers 32 consecutive entries of one row), element e = 2k + h of a
// thread is (row 4w + k, column lane + 32h).  L2 loads: the tile was written by another CTA
// of the same launch.
template <class TF>
__device__ __forceinline__ void tile_regs(const TF *src, int64_t ld, int64_t rows, TF v[8]) {
    const int lane = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int h = 0; h < 2; h++)
            v[2 * k + h] = r0 + k < rows ? __ldcg(src + (int64_t)(r0 + k) * ld + lane + 32 * h)
                                         : TF(0);
}
// dst[c][r] = the loaded tile's entry (r, c)
template <class TF>
__device__ __forceinline__ void tile_store_T(const TF v[8], TF (*dst)[kTileLd]) {
    const int lane = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * 4;
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int h = 0; h < 2; h++) dst[lane + 32 * h][r0 + k] = v[2 * k + h];
}
// dst[c][r] = src[r * ld + c] (r < rows, else 0), c < 64
template <class TF>
__device__ __forceinline__ void load_tile_T(const TF *src, int64_t ld, int64_t rows,
                                            TF (*dst)[kTileLd]) {
    TF v[8];
    tile_regs<TF>(src, ld, rows, v);
    tile_store_T<TF>(v, dst);
}

// acc[p][q] += sgn * sum_c bi[c][ty*2+p] bj[c][tx*4+q] (operands in transposed layout).
// The 64-term product is summed from zero and added to acc once: summing into acc
// directly would round every term at the magnitude of the (much larger) tile entry,
// which made the FP32 factor several times less accurate.
template <class TF, bool SUB>
__device__ __forceinline__ void tile_gemm_T(TF acc[2][4], const TF (*bi)[kTileLd],
                                            const TF (*bj)[kTileLd], int tx, int ty) {
    TF t[2][4];
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) t[p][q] = TF(0);
#pragma unroll 8
    for (int c = 0; c < NB; c++) {
        TF u[2], v[4];
        lds2<TF>(&bi[c][ty * 2], u);
        lds4<TF>(&bj[c][tx * 4], v);
#pragma unroll
        for (int p = 0; p < 2; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) t[p][q] = fma(u[p], v[q], t[p][q]);
    }
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = SUB ? acc[p][q] - t[p][q] : acc[p][q] + t[p][q];
}

// load tile (r0, c0) of A into acc (rows/columns beyond n: identity on the diagonal tile)
template <class TF>
__device__ __forceinline__ void load_acc(const TF *A, int64_t n, int64_t r0, int64_t c0,
                                         bool diag, TF acc[2][4], int tx, int ty) {
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int r = ty * 2 + p, c = tx * 4 + q;
            acc[p][q] = (r0 + r < n && c0 + c < n) ? __ldcg(&A[(r0 + r) * n + c0 + c])
                                                   : ((diag && r == c) ? TF(1) : TF(0));
        }
}

template <class TF>
__device__ __forceinline__ void store_acc(TF *A, int64_t n, int64_t r0, int64_t c0,
                                          const TF acc[2][4], int tx, int ty) {
#pragma unroll
    for (int p = 0; p < 2; p++) {
        const int r = ty * 2 + p;
        if (r0 + r >= n) continue;
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (c0 + tx * 4 + q < n) A[(r0 + r) * n + c0 + tx * 4 + q] = acc[p][q];
    }
}

// all threads' global stores of a tile are visible before its flag: the barrier orders
// them before thread 0's release, which is cumulative
__device__ __forceinline__ void publish(int *f) {
    __syncthreads();
    if (threadIdx.x == 0) st_release_gpu(f, 1);
}

template <class TF>
__device__ void chol_chain(TF *A, int64_t n, int nblk, TF *dinv, int *F, int *U, int *abort_w,
                           int32_t *err, unsigned char *smem_raw) {
    TF(*b0)[kTileLd] = reinterpret_cast<TF(*)[kTileLd]>(smem_raw);
    TF(*b1)[kTileLd] = b0 + NB;
    TF(*xt)[kTileLd] = b1 + NB;   // L_{j+1,j}^T (from the sub-solve, for the next update)
    TF(*at)[kTileLd] = xt + NB;   // A_{j+1,j}^T as the sub-solve reads it
    TF(*a_s)[NB + 1] = reinterpret_cast<TF(*)[NB + 1]>(&b0[0][0]);
    TF(*x_s)[NB + 1] = reinterpret_cast<TF(*)[NB + 1]>(&b1[0][0]);
    __shared__ int s_ok, s_pre;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    TF acc[2][4];   // the diagonal tile A~_jj of the coming step (loaded one step ahead)
    if (tid == 0) s_ok = wait_tile(&U[tile_id(0, 0)], abort_w, err);
    __syncthreads();
    if (!s_ok) return;
    load_acc<TF>(A, n, 0, 0, true, acc, tx, ty);
    for (int j = 0; j < nblk; j++) {
        const int64_t c0 = (int64_t)j * NB, r0 = c0 + NB;
        const bool next = j + 1 < nblk;
        if (j > 0) tile_gemm_T<TF, true>(acc, xt, xt, tx, ty);   // the update k = j - 1
#pragma unroll
        for (int p = 0; p < 2; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) a_s[ty * 2 + p][tx * 4 + q] = acc[p][q];
        __syncthreads();
        potrf_inv_smem<TF>(a_s, x_s, (int)min((int64_t)NB, n - c0), c0, err);
        if (next) {
            // L_{j+1,j} = A~_{j+1,j} L_jj^{-T}, computed transposed: xt = L_jj^{-1} A~_{j+1,j}^T
            // the next diagonal tile's flag is looked at now, beside this wait, and once more
            // after the sub-solve if it was not set yet
            if (tid == 0) s_ok = wait_tile(&U[tile_id(j + 1, j)], abort_w, err);
            if (tid == 32) s_pre = ld_acquire_gpu(&U[tile_id(j + 1, j + 1)]) != 0;
            __syncthreads();
            if (!s_ok) return;
            load_tile_T<TF>(A + r0 * n + c0, n, n - r0, at);   // at[k][r] = A_{j+1,j}[r][k]
            __syncthreads();
            TF o[2][4];
#pragma unroll
            for (int p = 0; p < 2; p++)
#pragma unroll
                for (int q = 0; q < 4; q++) o[p][q] = TF(0);
#pragma unroll 8
            for (int k = 0; k < NB; k++) {
                TF v[4];
                lds4<TF>(&at[k][tx * 4], v);
                const TF u0 = x_s[ty * 2][k], u1 = x_s[ty * 2 + 1][k];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    o[0][q] = fma(u0, v[q], o[0][q]);
                    o[1][q] = fma(u1, v[q], o[1][q]);
                }
            }
            // o[p][q] = L_{j+1,j}[tx*4+q][ty*2+p]; xt was last read by this step's update
#pragma unroll
            for (int p = 0; p < 2; p++) {
                TF *dst = &xt[ty * 2 + p][tx * 4];
                if constexpr (sizeof(TF) == 4) {
                    *reinterpret_cast<float4 *>(dst) = make_float4(o[p][0], o[p][1], o[p][2], o[p][3]);
                } else {
                    *reinterpret_cast<double2 *>(dst) = make_double2(o[p][0], o[p][1]);
                    *reinterpret_cast<double2 *>(dst + 2) = make_double2(o[p][2], o[p][3]);
                }
            }
            // the next diagonal tile goes into registers now if it is ready.  It is not
            // waited for here: its task may be queued behind tasks of this column that
            // wait for F(j, j), so the wait comes after the publication below.
            if (tid == 0 && !s_pre) s_pre = ld_acquire_gpu(&U[tile_id(j + 1, j + 1)]) != 0;
        }
        __syncthreads();   // xt complete; the next diagonal tile's flag seen
        const bool pre = next && s_pre;
        if (pre) load_acc<TF>(A, n, r0, r0, true, acc, tx, ty);
        // L_jj^{-1} into dinv, L_{j+1,j} into A: rows of 64, coalesced.  L_jj itself is not
        // stored: every solve with the factor applies L_jj^{-1}, so A's diagonal tiles keep
        // their last update.
        TF *Lj = dinv + (int64_t)j * NB * NB;
        for (int e = tid; e < NB * NB; e += blockDim.x) {
            const int i = e >> 6, c = e & 63;
            Lj[e] = x_s[i][c];
            if (next && r0 + i < n) A[(r0 + i) * n + c0 + c] = xt[c][i];
        }
        __syncthreads();   // every store is issued before the (cumulative) releases
        if (tid == 0) {
            st_release_gpu(&F[tile_id(j, j)], 1);
            if (next) st_release_gpu(&F[tile_id(j + 1, j)], 1);
        }
        if (next && !pre) {
            if (tid == 0) s_ok = wait_tile(&U[tile_id(j + 1, j + 1)], abort_w, err);
            __syncthreads();
            if (!s_ok) return;
            load_acc<TF>(A, n, r0, r0, true, acc, tx, ty);
        }
    }
}

template <class TF>
__global__ void __launch_bounds__(512, 1) k_chol_tiles(TF *A, int64_t n, int nblk, TF *dinv,
                                                       int *flags, int32_t *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TF(*b0)[kTileLd] = reinterpret_cast<TF(*)[kTileLd]>(smem_raw);
    TF(*b1)[kTileLd] = b0 + NB;
    __shared__ int s_task, s_ok, s_fa, s_fb, s_pa[2], s_pb[2];
    const int ntask = nblk * (nblk + 1) / 2;
    int *F = flags, *U = flags + ntask, *ticket = flags + 2 * ntask, *abort_w = ticket + 1;
    if (blockIdx.x == 0) {
        chol_chain<TF>(A, n, nblk, dinv, F, U, abort_w, err, smem_raw);
        return;
    }
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;   // rows ty*2+{0,1}, cols tx*4+{0..3}
    for (;;) {
        if (tid == 0) s_task = atomicAdd(ticket, 1);
        __syncthreads();
        const int t = s_task;
        if (t >= ntask) return;
        int j = 0, rem = t;
        while (rem >= nblk - j) { rem -= nblk - j; j++; }
        const int i = j + rem;
        const int64_t r0 = (int64_t)i * NB, c0 = (int64_t)j * NB;
        const int64_t rows_i = n - r0;
        const int kmax = i == j ? max(j - 1, 0) : j;   // the chain applies k = j - 1 to (j, j)
        TF acc[2][4];
        load_acc<TF>(A, n, r0, c0, false, acc, tx, ty);
        // Updates k = 0 .. kmax-1, pipelined: the tiles L_ik, L_jk of update k + 1 are
        // loaded into registers while update k's product runs (when their flags are
        // already set; otherwise after it, with a blocking wait), and stored into the other
        // pair of shared tiles.  Threads 0 and 32 read the two flags at the same time.
        TF va[8], vb[8];
        bool have = false;   // va / vb hold the tiles of update k
        for (int k = 0; k < kmax; k++) {
            TF(*ta)[kTileLd] = b0 + (k & 1) * 2 * NB;
            TF(*tb)[kTileLd] = ta + NB;
            if (!have) {
                if (tid == 0) s_fa = wait_tile(&F[tile_id(i, k)], abort_w, err);
                if (tid == 32) s_fb = wait_tile(&F[tile_id(j, k)], abort_w, err);
                __syncthreads();
                if (!(s_fa && s_fb)) return;
                tile_regs<TF>(A + r0 * n + (int64_t)k * NB, n, rows_i, va);
                if (i != j) tile_regs<TF>(A + c0 * n + (int64_t)k * NB, n, n - c0, vb);
            }
            tile_store_T<TF>(va, ta);
            if (i != j) tile_store_T<TF>(vb, tb);
            const int q = (k + 1) & 1;
            if (k + 1 < kmax) {   // a look at update k + 1's flags, without waiting
                if (tid == 0) s_pa[q] = ld_acquire_gpu(&F[tile_id(i, k + 1)]) != 0;
                if (tid == 32) s_pb[q] = ld_acquire_gpu(&F[tile_id(j, k + 1)]) != 0;
            }
            __syncthreads();   // update k's tiles stored (the pair written two updates ago
                               // is no longer read); update k + 1's flags seen
            have = k + 1 < kmax && s_pa[q] && s_pb[q];
            if (have) {
                tile_regs<TF>(A + r0 * n + (int64_t)(k + 1) * NB, n, rows_i, va);
                if (i != j) tile_regs<TF>(A + c0 * n + (int64_t)(k + 1) * NB, n, n - c0, vb);
            }
            tile_gemm_T<TF, true>(acc, ta, i == j ? ta : tb, tx, ty);
        }
        __syncthreads();   // the last product is done before the shared tiles are reused
        if (i <= j + 1) {
            // diagonal or sub-diagonal tile: the chain finishes it
            store_acc<TF>(A, n, r0, c0, acc, tx, ty);
            publish(&U[tile_id(i, j)]);
            continue;
        }
        // L_ij = A_ij L_jj^{-T}: o[p][q] = sum_c acc[ty*2+p][c] Linv[tx*4+q][c]
        TF(*a)[NB + 1] = reinterpret_cast<TF(*)[NB + 1]>(smem_raw);   // overlays b0 only
#pragma unroll
        for (int p = 0; p < 2; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) a[ty * 2 + p][tx * 4 + q] = acc[p][q];
        if (tid == 0) s_ok = wait_tile(&F[tile_id(j, j)], abort_w, err);
        __syncthreads();
        if (!s_ok) return;
        load_tile_T<TF>(dinv + (int64_t)j * NB * NB, NB, NB, b1);   // b1[c][q] = Linv[q][c]
        __syncthreads();
        TF o[2][4];
#pragma unroll
        for (int p = 0; p < 2; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) o[p][q] = TF(0);
#pragma unroll 8
        for (int c = 0; c < NB; c++) {
            TF v[4];
            lds4<TF>(&b1[c][tx * 4], v);
            const TF u0 = a[ty * 2][c], u1 = a[ty * 2 + 1][c];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                o[0][q] = fma(u0, v[q], o[0][q]);
                o[1][q] = fma(u1, v[q], o[1][q]);
            }
        }
        store_acc<TF>(A, n, r0, c0, o, tx, ty);
        publish(&F[tile_id(i, j)]);
    }
}

// at most this many right-hand sides per triangular-solve launch
constexpr int kMaxRhs = 24;

// ---------------------------------------------------------------------------------
// Batched block-step triangular solves across meshes (no waiting between CTAs, so the
// meshes of a batch share launches).  Step s: mesh m solves its block k = s (forward)
// or nblk_m - 1 - s (backward) with the diagonal inverse, then updates the blocks that
// depend on it.  All right-hand sides of a mesh (<= 24, column-major, ld = n) together.
// ---------------------------------------------------------------------------------
template <class TF>
__global__ void __launch_bounds__(256) k_btrsm_diag(const BatchTrsmDesc *__restrict__ d, int s,
                                                    int nrhs, int backward) {
    __shared__ TF dv[NB][NB + 1];
    __shared__ TF tt[NB][kMaxRhs + 1];
    const BatchTrsmDesc &D = d[blockIdx.x];
    if (!D.active || s >= D.nblk) return;
    const int k = backward ? D.nblk - 1 - s : s;
    const int64_t n = D.n, r0 = (int64_t)k * NB;
    const int nb = (int)min((int64_t)NB, n - r0);
    const TF *Dinv = reinterpret_cast<const TF *>(D.dinv) + (int64_t)k * NB * NB;
    TF *Y = reinterpret_cast<TF *>(D.y);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) dv[e >> 6][e & 63] = Dinv[e];
    for (int e = threadIdx.x; e < NB * nrhs; e += blockDim.x) {
        const int r = e & 63, c = e >> 6;
        tt[r][c] = r < nb ? Y[(int64_t)c * n + r0 + r] : TF(0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * nrhs; e += blockDim.x) {
        const int r = e & 63, c = e >> 6;
        TF acc = TF(0);
        if (!backward)
            for (int q = 0; q <= r; q++) acc += dv[r][q] * tt[q][c];
        else
            for (int q = r; q < NB; q++) acc += dv[q][r] * tt[q][c];
        if (r < nb) Y[(int64_t)c * n + r0 + r] = acc;
    }
}

template <class TF>
__global__ void __launch_bounds__(256) k_btrsm_update(const BatchTrsmDesc *__restrict__ d, int s,
                                                      int nrhs, int backward) {
    __shared__ TF lt[NB][NB + 1];
    __shared__ TF xs[NB][kMaxRhs + 1];
    const BatchTrsmDesc &D = d[blockIdx.y];
    if (!D.active || s >= D.nblk) return;
    const int k = backward ? D.nblk - 1 - s : s;
    const int i = backward ? k - 1 - (int)blockIdx.x : k + 1 + (int)blockIdx.x;
    if (i < 0 || i >= D.nblk) return;
    const int64_t n = D.n, r0 = (int64_t)i * NB, c0 = (int64_t)k * NB;
    const int nb = (int)min((int64_t)NB, n - r0), nk = (int)min((int64_t)NB, n - c0);
    const TF *L = reinterpret_cast<const TF *>(D.L);
    TF *Y = reinterpret_cast<TF *>(D.y);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int a = e >> 6, b = e & 63;
        if (!backward) {   // lt[r][q] = L[r0 + r][c0 + q]
            lt[a][b] = (a < nb && b < nk) ? L[(r0 + a) * n + c0 + b] : TF(0);
        } else {           // lt[r][q] = L[c0 + q][r0 + r]
            lt[b][a] = (a < nk && b < nb) ? L[(c0 + a) * n + r0 + b] : TF(0);
        }
    }
    for (int e = threadIdx.x; e < NB * nrhs; e += blockDim.x) {
        const int q = e & 63, c = e >> 6;
        xs[q][c] = q < nk ? Y[(int64_t)c * n + c0 + q] : TF(0);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * nrhs; e += blockDim.x) {
        const int r = e & 63, c = e >> 6;
        TF acc = TF(0);
#pragma unroll 8
        for (int q = 0; q < NB; q++) acc += lt[r][q] * xs[q][c];
        if (r < nb) Y[(int64_t)c * n + r0 + r] -= acc;
    }
}

template <class TF>
int chol_tiles_t(TF *A, int64_t n, cudaStream_t s, Mesh *m) {
    if (n <= 0) return FEM3_OK;
    const int nblk = (int)((n + NB - 1) / NB);
    const int ntask = nblk * (nblk + 1) / 2;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        FEM3_CUDA(cudaGetDevice(&dev));
        FEM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    FEM3_CUDA(cudaMemsetAsync(m->chol_flags, 0, sizeof(int32_t) * (2 * ntask + 2), s));
    // one CTA per SM: the chain CTA gets an SM of its own
    const int grid = std::min(ntask + 1, std::max(sms, 2));
    kc_begin(m, KC_FACTOR);
    k_chol_tiles<TF><<<grid, 512, kCholTilesSmem * sizeof(TF), s>>>(
        A, n, nblk, reinterpret_cast<TF *>(m->dinv), m->chol_flags, m->err);
    kc_end(m, KC_FACTOR);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// ---------------------------------------------------------------------------------
// Chain triangular solves (one launch per direction, 1..24 right-hand sides).
// Forward: y_j = Dinv_j (b_j - sum_{k<j} L_jk y_k); backward: x_j = Dinv_j^T (y_j -
// sum_{k>j} L_kj^T x_k).  Step s solves block j(s) (j = s forward, nblk-1-s backward);
// M(s, s') is the coefficient tile between the blocks of steps s and s' < s.
// CTA 0 runs the chain: at step s it waits for the workers' partial sum S_s (all
// dependencies s' < s - D), applies the D nearest tiles M(s, s-1 .. s-D) itself from
// registers loaded one step ahead, multiplies by the diagonal inverse and publishes the
// block (flag Yf).  Worker CTAs take steps s > D from an atomic ticket in increasing order,
// accumulate S_s as the blocks s' <= s - D - 1 appear and publish it (flag Pf).  The
// chain only waits for tickets that precede the ones any worker can be blocked on, so the
// launch needs no co-residency; waits are bounded (ERR_SOLVE, abort word).
// Y is column-major (n x nrhs, leading dimension n), solved in place.  flags: Yf [nblk],
// Pf [nblk], ticket, abort word, all zero at launch; Z: nblk x 64 x 24 workspace.
// ---------------------------------------------------------------------------------
constexpr int kSolveThreads = 512;            // thread (r, g): row r = t & 63, column chunk g = t >> 6

template <class TF> struct SolveCfg {
    // dependency tiles the chain applies itself: one more lengthens every chain step, one
    // fewer puts the workers' hand-over on the critical path (2 timed fastest, both types)
    static constexpr int D = 2;
};

// shared memory: ring of D + 1 solved blocks [64][NR] (chain) or one dependency block and
// one right-hand-side block (worker), and 8 partial buffers [64][NR + 1]
template <class TF, int NR>
constexpr size_t solve_chain_smem() {
    return ((size_t)(SolveCfg<TF>::D + 1) * NB * NR + (size_t)8 * NB * (NR + 1)) * sizeof(TF);
}

// Precomputed chain operators.  Step s of a direction solves block j; its dependency d
// (d < D) is the block solved at step s - 1 - d.  G(s, d) = Dm_j M(s, s-1-d), with Dm_j
// the diagonal inverse as applied (transposed when backward) and M the coefficient tile,
// so that the chain step is y_s = z_s - sum_d G(s, d) y_{s-1-d}, z_s = Dm_j (b_s - S_s).
// Layout per (direction, s, d): element (r, c = 8g + e) at (g * 64 + r) * 8 + e, i.e. the
// eight values thread (r, g) needs are 32 contiguous bytes.
__device__ __forceinline__ int64_t gop_index(int dir, int s, int d, int nblk, int D) {
    return (((int64_t)dir * nblk + s) * D + d) * (NB * NB);
}

__device__ __forceinline__ int solve_blk(int s, int nblk, bool backward) {
    return backward ? nblk - 1 - s : s;
}

// NR consecutive values of a shared row (16-byte aligned when NR > 1)
template <class TF, int NR>
__device__ __forceinline__ void ld_row(const TF *p, TF out[NR]) {
    if constexpr (NR == 1) {
        out[0] = p[0];
    } else if constexpr (sizeof(TF) == 4) {
#pragma unroll
        for (int k = 0; k < NR / 4; k++) {
            const float4 q = reinterpret_cast<const float4 *>(p)[k];
            out[4 * k] = q.x; out[4 * k + 1] = q.y; out[4 * k + 2] = q.z; out[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < NR / 2; k++) {
            const double2 q = reinterpret_cast<const double2 *>(p)[k];
            out[2 * k] = q.x; out[2 * k + 1] = q.y;
        }
    }
}

// this thread's eight entries M[r][8g .. 8g+7] of the tile between blocks j (solved) and jd
template <class TF>
__device__ __forceinline__ void load_coef(const TF *__restrict__ L, int64_t n, int j, int jd,
                                          bool backward, int r, int g, TF out[8]) {
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int c = g * 8 + e;
        const int64_t row = backward ? (int64_t)jd * NB + c : (int64_t)j * NB + r;
        const int64_t col = backward ? (int64_t)j * NB + r : (int64_t)jd * NB + c;
        out[e] = row < n ? __ldg(&L[row * n + col]) : TF(0);
    }
}

// diagonal inverse of block j as applied at this step (transposed when backward)
template <class TF>
__device__ __forceinline__ void load_dinv(const TF *__restrict__ Dinv, int j, bool backward, int r,
                                          int g, TF out[8]) {
    const TF *Dj = Dinv + (int64_t)j * NB * NB;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const int c = g * 8 + e;
        out[e] = __ldg(&Dj[backward ? c * NB + r : r * NB + c]);
    }
}

__device__ __forceinline__ bool wait_flag(const int *f, int *abort_w, int32_t *err) {
    int spins = 0;
    while (ld_acquire_gpu(f) == 0) {
        if (ld_acquire_gpu(abort_w) != 0) return false;
        if (++spins > kSpinLimit) {
            atomicAdd(&err[ERR_SOLVE], 1);
            atomicExch(abort_w, 1);
            return false;
        }
        if (spins > 64) __nanosleep(32);
    }
    return true;
}

// part[v] += sum_e m[e] rows[8g + e][v], v < NR
template <class TF, int NR>
__device__ __forceinline__ void chunk_gemv(const TF m[8], const TF *rows, int g, TF part[NR]) {
#pragma unroll
    for (int e = 0; e < 8; e++) {
        TF yv[NR];
        ld_row<TF, NR>(rows + (g * 8 + e) * NR, yv);
#pragma unroll
        for (int v = 0; v < NR; v++) part[v] = fma(m[e], yv[v], part[v]);
    }
}

// red[g][r][v] = part[v]; after a barrier, the owner of (r, v) adds the eight partials
template <class TF, int NR>
__device__ __forceinline__ void store_partial(TF *red, int r, int g, const TF part[NR]) {
#pragma unroll
    for (int v = 0; v < NR; v++) red[(g * NB + r) * (NR + 1) + v] = part[v];
}
template <class TF, int NR>
__device__ __forceinline__ TF sum_partials(const TF *red, int r, int v) {
    TF t = TF(0);
#pragma unroll
    for (int q = 0; q < 8; q++) t += red[(q * NB + r) * (NR + 1) + v];
    return t;
}

// G(s, d) for one direction, step and dependency (grid: nblk x D x 2 directions)
template <class TF>
__global__ void __launch_bounds__(256) k_solve_prep(const TF *__restrict__ L,
                                                    const TF *__restrict__ Dinv, int64_t n,
                                                    int nblk, TF *Gop) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int D = SolveCfg<TF>::D;
    TF(*dm)[NB + 1] = reinterpret_cast<TF(*)[NB + 1]>(smem_raw);   // Dm[r][k]
    TF(*mm)[NB + 1] = dm + NB;                                     // M[k][c]
    const int s = blockIdx.x, d = blockIdx.y, dir = blockIdx.z;
    if (s - 1 - d < 0) return;
    const bool bw = dir != 0;
    const int j = solve_blk(s, nblk, bw), jd = solve_blk(s - 1 - d, nblk, bw);
    const TF *Dj = Dinv + (int64_t)j * NB * NB;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int hi = e >> 6, lo = e & 63;
        // Dm[r][k] = Dinv_j[r][k] (forward) or Dinv_j[k][r] (backward); read row-major
        if (!bw) dm[hi][lo] = Dj[e];
        else dm[lo][hi] = Dj[e];
        // M[k][c] = L[j*64 + k][jd*64 + c] (forward) or L[jd*64 + c][j*64 + k] (backward)
        const int64_t grow = (bw ? (int64_t)jd : (int64_t)j) * NB + hi;
        const int64_t gcol = (bw ? (int64_t)j : (int64_t)jd) * NB + lo;
        const TF v = grow < n ? L[grow * n + gcol] : TF(0);
        if (!bw) mm[hi][lo] = v;
        else mm[lo][hi] = v;
    }
    __syncthreads();
    TF *G = Gop + gop_index(dir, s, d, nblk, D);
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e & 63, c = e >> 6;
        TF acc = TF(0);
#pragma unroll 8
        for (int k = 0; k < NB; k++) acc = fma(dm[r][k], mm[k][c], acc);
        G[((c >> 3) * NB + r) * 8 + (c & 7)] = acc;
    }
}

template <class TF>
__device__ __forceinline__ void load_g(const TF *G, int r, int g, TF out[8]) {
    const TF *p = G + (g * NB + r) * 8;
    if constexpr (sizeof(TF) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
        out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + k);
            out[2 * k] = a.x; out[2 * k + 1] = a.y;
        }
    }
}

template <class TF, int NR>
__device__ void solve_chain(int64_t n, int nblk, TF *Y, int nrhs, bool backward, const TF *Gop,
                            const TF *Z, int *Yf, const int *Pf, int *abort_w, int32_t *err,
                            unsigned char *smem_raw) {
    constexpr int D = SolveCfg<TF>::D;
    TF *yr = reinterpret_cast<TF *>(smem_raw);        // [D + 1][64][NR] ring of solved blocks
    TF *red = yr + (D + 1) * NB * NR;                 // [8][64][NR + 1]
    __shared__ int s_ok;
    const int tid = threadIdx.x, r = tid & 63, g = tid >> 6;
    const int dir = backward ? 1 : 0;
    TF gc[D][8], gn[D][8];
#pragma unroll
    for (int d = 0; d < D; d++)
#pragma unroll
        for (int e = 0; e < 8; e++) { gc[d][e] = TF(0); gn[d][e] = TF(0); }
    for (int s = 0; s < nblk; s++) {
        const int j = solve_blk(s, nblk, backward);
        const int64_t row = (int64_t)j * NB + r;
        // warp 1 waits for z_s while thread 0 may still be publishing the last block
        if (tid == 32) s_ok = wait_flag(&Pf[s], abort_w, err);
        if (s + 1 < nblk) {
#pragma unroll
            for (int d = 0; d < D; d++)
                if (s - d >= 0) load_g<TF>(Gop + gop_index(dir, s + 1, d, nblk, D), r, g, gn[d]);
        }
        TF part[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) part[v] = TF(0);
#pragma unroll
        for (int d = 0; d < D; d++)
            if (s - 1 - d >= 0)
                chunk_gemv<TF, NR>(gc[d], yr + ((s - 1 - d) % (D + 1)) * NB * NR, g, part);
        store_partial<TF, NR>(red, r, g, part);
        __syncthreads();
        if (!s_ok) return;
        TF *ys = yr + (s % (D + 1)) * NB * NR;
#pragma unroll
        for (int h = 0; h < (NR + 7) / 8; h++) {
            const int v = g + 8 * h;
            if (v < NR) {
                const TF y = __ldcg(&Z[((int64_t)s * NB + r) * kMaxRhs + v]) -
                             sum_partials<TF, NR>(red, r, v);
                ys[r * NR + v] = y;
                if (row < n && v < nrhs) Y[row + (int64_t)v * n] = y;
            }
        }
        __syncthreads();
        // the barrier orders every thread's stores of the block before thread 0's release,
        // which carries them to the consumers that acquire the flag (release is cumulative)
        if (tid == 0) st_release_gpu(&Yf[s], 1);
#pragma unroll
        for (int d = 0; d < D; d++)
#pragma unroll
            for (int e = 0; e < 8; e++) gc[d][e] = gn[d][e];
    }
}

template <class TF, int NR>
__global__ void __launch_bounds__(kSolveThreads, 1) k_solve_chain(
    const TF *__restrict__ L, const TF *__restrict__ Dinv, int64_t n, int nblk, TF *Y, int nrhs,
    int backward, const TF *__restrict__ Gop, TF *Z, int *flags, int32_t *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int D = SolveCfg<TF>::D;
    int *Yf = flags, *Pf = flags + nblk, *ticket = flags + 2 * nblk, *abort_w = ticket + 1;
    if (blockIdx.x == 0) {
        solve_chain<TF, NR>(n, nblk, Y, nrhs, backward != 0, Gop, Z, Yf, Pf, abort_w, err, smem_raw);
        return;
    }
    TF *yb = reinterpret_cast<TF *>(smem_raw);   // [2][64][NR] dependency blocks, then b - S
    TF *red = yb + 2 * NB * NR;                  // [8][64][NR + 1]
    __shared__ int s_task, s_ok, s_pre[2];
    const int tid = threadIdx.x, r = tid & 63, g = tid >> 6;
    const bool bw = backward != 0;
    for (;;) {
        if (tid == 0) s_task = atomicAdd(ticket, 1);
        __syncthreads();
        const int s = s_task;
        if (s >= nblk) return;
        const int j = solve_blk(s, nblk, bw);
        TF part[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) part[v] = TF(0);
        // Dependencies sd = 0 .. last, pipelined: the solved block y_{sd+1} is loaded into
        // registers while the product with y_sd runs (when its flag is already set;
        // otherwise after it, with a blocking wait) and stored into the other shared buffer.
        constexpr int PY = (NB * NR + kSolveThreads - 1) / kSolveThreads;   // y values / thread
        const int last = s - D - 1;
        auto load_y = [&](int sd, TF yv[PY]) {
            const int jd = solve_blk(sd, nblk, bw);
#pragma unroll
            for (int k = 0; k < PY; k++) {
                const int e = tid + k * kSolveThreads;
                const int c = e / NR, v = e % NR;
                const int64_t rr = (int64_t)jd * NB + c;
                yv[k] = (e < NB * NR && rr < n && v < nrhs) ? __ldcg(&Y[rr + (int64_t)v * n]) : TF(0);
            }
        };
        TF tc[8], yv[PY];
        bool have = false;   // yv holds y_sd
        if (last >= 0) load_coef<TF>(L, n, j, solve_blk(0, nblk, bw), bw, r, g, tc);
        for (int sd = 0; sd <= last; sd++) {
            TF *ybs = yb + (sd & 1) * NB * NR;
            if (!have) {
                if (tid == 0) s_ok = wait_flag(&Yf[sd], abort_w, err);
                __syncthreads();
                if (!s_ok) return;
                load_y(sd, yv);
            }
#pragma unroll
            for (int k = 0; k < PY; k++)
                if (tid + k * kSolveThreads < NB * NR) ybs[tid + k * kSolveThreads] = yv[k];
            const int q = (sd + 1) & 1;
            if (tid == 0 && sd + 1 <= last) s_pre[q] = ld_acquire_gpu(&Yf[sd + 1]) != 0;
            __syncthreads();   // y_sd stored (the buffer written two dependencies ago is no
                               // longer read); y_{sd+1}'s flag seen
            have = sd + 1 <= last && s_pre[q];
            if (have) load_y(sd + 1, yv);
            TF tn[8];
            if (sd + 1 <= last) load_coef<TF>(L, n, j, solve_blk(sd + 1, nblk, bw), bw, r, g, tn);
            chunk_gemv<TF, NR>(tc, ybs, g, part);
#pragma unroll
            for (int e = 0; e < 8; e++) tc[e] = tn[e];
        }
        __syncthreads();   // the last product is done before yb is reused
        // t = b_s - S_s into yb, then z_s = Dm_j t
        store_partial<TF, NR>(red, r, g, part);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < (NR + 7) / 8; h++) {
            const int v = g + 8 * h;
            if (v < NR) {
                const int64_t row = (int64_t)j * NB + r;
                const TF b = (row < n && v < nrhs) ? __ldcg(&Y[row + (int64_t)v * n]) : TF(0);
                yb[r * NR + v] = b - sum_partials<TF, NR>(red, r, v);
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NR; v++) part[v] = TF(0);
        {
            TF dm[8];
            load_dinv<TF>(Dinv, j, bw, r, g, dm);
            chunk_gemv<TF, NR>(dm, yb, g, part);
        }
        store_partial<TF, NR>(red, r, g, part);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < (NR + 7) / 8; h++) {
            const int v = g + 8 * h;
            if (v < NR) Z[((int64_t)s * NB + r) * kMaxRhs + v] = sum_partials<TF, NR>(red, r, v);
        }
        __syncthreads();
        if (tid == 0) st_release_gpu(&Pf[s], 1);
    }
}

template <class TF, int NR>
static int launch_solve_chain(const TF *L, const TF *Dinv, int64_t n, int nblk, TF *Y, int nrhs,
                              const TF *Gop, TF *Z, int workers, cudaStream_t s, Mesh *m) {
    static bool attr = false;
    if (!attr) {
        FEM3_CUDA(cudaFuncSetAttribute(k_solve_chain<TF, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)solve_chain_smem<TF, NR>()));
        attr = true;
    }
    for (int backward = 0; backward < 2; backward++) {
        FEM3_CUDA(cudaMemsetAsync(m->flags, 0, sizeof(int32_t) * (2 * nblk + 2), s));
        kc_begin(m, KC_CHAIN);
        k_solve_chain<TF, NR><<<1 + workers, kSolveThreads, solve_chain_smem<TF, NR>(), s>>>(
            L, Dinv, n, nblk, Y, nrhs, backward, Gop, Z, m->flags, m->err);
        kc_end(m, KC_CHAIN);
        note_launch(m);
    }
    return FEM3_OK;
}

// Chain operators of the current factor (run once per factorisation).
template <class TF>
int solve_prep_t(const TF *L, int64_t n, cudaStream_t s, Mesh *m) {
    if (n <= 0) return FEM3_OK;
    const int nblk = (int)((n + NB - 1) / NB);
    const size_t sh = 2 * NB * (NB + 1) * sizeof(TF);
    static bool attr = false;
    if (!attr) {
        FEM3_CUDA(cudaFuncSetAttribute(k_solve_prep<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        attr = true;
    }
    k_solve_prep<TF><<<dim3(nblk, SolveCfg<TF>::D, 2), 256, sh, s>>>(
        L, reinterpret_cast<const TF *>(m->dinv), n, nblk, reinterpret_cast<TF *>(m->solve_G));
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// L y = b (forward) then L^T x = y (backward), in place in Y (n x nrhs, nrhs <= 24);
// uses the operators of solve_prep_t for the same factor.
template <class TF>
int solve_chain_t(const TF *L, int64_t n, TF *Y, int nrhs, cudaStream_t s, Mesh *m) {
    if (n <= 0) return FEM3_OK;
    if (nrhs < 1 || nrhs > kMaxRhs) return set_error(FEM3_E_ARG, "1..24 right-hand sides per block solve");
    const int nblk = (int)((n + NB - 1) / NB);
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        FEM3_CUDA(cudaGetDevice(&dev));
        FEM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int workers = std::max(1, std::min(nblk, sms - 1));
    const TF *Dinv = reinterpret_cast<const TF *>(m->dinv);
    const TF *Gop = reinterpret_cast<const TF *>(m->solve_G);
    TF *Z = reinterpret_cast<TF *>(m->solve_ws);
    if (nrhs == 1) FEM3_TRY((launch_solve_chain<TF, 1>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    else if (nrhs <= 4) FEM3_TRY((launch_solve_chain<TF, 4>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    else if (nrhs <= 8) FEM3_TRY((launch_solve_chain<TF, 8>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    else if (nrhs <= 16) FEM3_TRY((launch_solve_chain<TF, 16>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    else if (nrhs <= 20) FEM3_TRY((launch_solve_chain<TF, 20>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    else FEM3_TRY((launch_solve_chain<TF, 24>(L, Dinv, n, nblk, Y, nrhs, Gop, Z, workers, s, m)));
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// L y = b then L^T x = y, in place; cooperative wavefront kernel when all block CTAs
// fit on the device at once, otherwise blocked substitution with one launch per block.
template <class TF>
int trsv_t(const TF *L, int64_t n, TF *y, cudaStream_t s, Mesh *m) {
    return solve_chain_t<TF>(L, n, y, 1, s, m);
}

// per-axis forms sum_g w_g ((L lam)(R u) + (R lam)(L u)) (adjoint), one CTA per bin
__global__ void __launch_bounds__(256) k_axis_form(
    const float2 *__restrict__ tabL, const float2 *__restrict__ tabR,
    const int32_t *__restrict__ gp_off, const int32_t *__restrict__ gp_idx,
    const int32_t *__restrict__ dof_off, const int32_t *__restrict__ dof_idx,
    const int64_t *__restrict__ tab_off, const int32_t *__restrict__ tab_ld,
    const double *__restrict__ gw, const double *__restrict__ u, const double *__restrict__ lam,
    double *out) {
    extern __shared__ double sm[];
    const int bin = blockIdx.x;
    const int D = dof_off[bin + 1] - dof_off[bin];
    const int G = gp_off[bin + 1] - gp_off[bin];
    if (D == 0 || G == 0) return;
    const int ld = tab_ld[bin];
    const float2 *L = tabL + tab_off[bin], *R = tabR + tab_off[bin];
    const int32_t *dofs = dof_idx + dof_off[bin];
    const int32_t *slots = gp_idx + gp_off[bin];
    double *ub = sm, *lb = sm + D;
    __shared__ double red[8];
    for (int c = threadIdx.x; c < D; c += blockDim.x) { ub[c] = u[dofs[c]]; lb[c] = lam[dofs[c]]; }
    __syncthreads();
    double acc = 0;
    for (int r = threadIdx.x; r < G; r += blockDim.x) {
        double Lu = 0, Ru = 0, Ll = 0, Rl = 0;
        for (int c = 0; c < D; c++) {
            const float2 lp = L[(int64_t)c * ld + r], rp = R[(int64_t)c * ld + r];
            const double lv = (double)lp.x + (double)lp.y, rv = (double)rp.x + (double)rp.y;
            Lu = fma(lv, ub[c], Lu); Ru = fma(rv, ub[c], Ru);
            Ll = fma(lv, lb[c], Ll); Rl = fma(rv, lb[c], Rl);
        }
        acc += gw[slots[r]] * (Ll * Ru + Rl * Lu);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        atomicAdd(out, s);
    }
}

// r = b - Au; norms[0] += |r|^2, norms[1] += |b|^2
__global__ void k_residual(const double *__restrict__ b, const double *__restrict__ Au, int64_t n,
                           double *r, double *norms) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0, bb = 0;
    if (i < n) {
        double v = b[i] - Au[i];
        r[i] = v;
        rr = v * v;
        bb = b[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&norms[0], rr);
        atomicAdd(&norms[1], bb);
    }
}

// r = b - Au for column blockIdx.y; norms[2c] += |r_c|^2, norms[2c+1] += |b_c|^2
__global__ void k_residual_cols(const double *__restrict__ b, const double *__restrict__ Au,
                                int64_t n, double *r, double *norms) {
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

// r -= Ad (the late sweeps' residual update) with the norms of r and b per column
__global__ void k_residual_update_cols(const double *__restrict__ b, const double *__restrict__ Ad,
                                       int64_t n, double *r, double *norms) {
    const int c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0, bb = 0;
    if (i < n) {
        const int64_t k = (int64_t)c * n + i;
        const double v = r[k] - Ad[k];
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

__global__ void k_f32_to_f64_n(const float *__restrict__ a, double *b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

// ui[i][v] = u[v * n + i] for v < nv, zero for nv <= v < NR (NR = 4 or 8 vectors a pass)
template <int NR>
__global__ void k_interleave(const double *__restrict__ u, int64_t n, int nv, double *ui) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NR * n) return;
    const int64_t i = e / NR;
    const int v = (int)(e - i * NR);
    ui[e] = v < nv ? u[(int64_t)v * n + i] : 0.0;
}

__global__ void k_to_f32(const double *__restrict__ a, float *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_axpy_f32(const float *__restrict__ d, double *u, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) u[i] += (double)d[i];
}
__global__ void k_f32_to_f64(const float *__restrict__ a, double *b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

__global__ void k_sub(const double *__restrict__ a, const double *__restrict__ b, double *c,
                      int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) c[i] = a[i] - b[i];
}

inline unsigned g256(int64_t n) { return (unsigned)(n > 0 ? (n + 255) / 256 : 1); }

}  // namespace

// upper triangle := transpose of the lower triangle (n x n row-major)
__global__ void k_sym_from_lower(double *A, int64_t n) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int64_t i = e / n, j = e % n;
    if (j > i) A[e] = A[j * n + i];
}

int sym_from_lower(double *A, int64_t n, cudaStream_t s) {
    k_sym_from_lower<<<g256(n * n), 256, 0, s>>>(A, n);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int f32_to_f64(const float *a, double *b, int64_t n, cudaStream_t s) {
    k_f32_to_f64<<<g256(n), 256, 0, s>>>(a, b, n);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int sub_vec(const double *a, const double *b, double *c, int64_t n, cudaStream_t s) {
    k_sub<<<g256(n), 256, 0, s>>>(a, b, c, n);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int residual_norm(Mesh *m, const double *b, const double *Au, double *rel) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    FEM3_CUDA(cudaMemsetAsync(m->norms, 0, sizeof(double) * 2, s));
    k_residual<<<g256(n), 256, 0, s>>>(b, Au, n, m->vec64[1], m->norms);
    note_launch(m);
    FEM3_CUDA(cudaMemcpyAsync(m->h_norms, m->norms, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    *rel = m->h_norms[1] > 0 ? sqrt(m->h_norms[0] / m->h_norms[1]) : 0.0;
    return FEM3_OK;
}

// L Y = B then L^T X = Y for nrhs <= 24 columns (column-major, leading dimension n)
template <class TF>
int trsm_t(const TF *L, int64_t n, TF *Y, int nrhs, cudaStream_t s, Mesh *m) {
    return solve_chain_t<TF>(L, n, Y, nrhs, s, m);
}

// Forward then backward block-step sweeps over all meshes of a batch (descriptors in
// device memory, nrhs <= 16, max_nblk = largest block count).
template <class TF>
int trsm_batch_t(const BatchTrsmDesc *d_desc, int n_mesh, int max_nblk, int nrhs, cudaStream_t s) {
    for (int backward = 0; backward < 2; backward++)
        for (int st = 0; st < max_nblk; st++) {
            k_btrsm_diag<TF><<<n_mesh, 256, 0, s>>>(d_desc, st, nrhs, backward);
            if (st + 1 < max_nblk)
                k_btrsm_update<TF><<<dim3(max_nblk - 1 - st, n_mesh), 256, 0, s>>>(d_desc, st, nrhs,
                                                                                   backward);
        }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int trsm_batch(const BatchTrsmDesc *d_desc, int n_mesh, int max_nblk, int nrhs, bool fp64,
               cudaStream_t s) {
    return fp64 ? trsm_batch_t<double>(d_desc, n_mesh, max_nblk, nrhs, s)
                : trsm_batch_t<float>(d_desc, n_mesh, max_nblk, nrhs, s);
}

int load_vector(Mesh *m, const double *f_d, int nrhs, double *b_d) {
    cudaStream_t s = m->stream;
    FEM3_CUDA(cudaMemsetAsync(b_d, 0, sizeof(double) * m->n_dof * nrhs, s));
    k_load<<<g256(m->n_tets), 256, 0, s>>>(m->tets, m->vol, m->dof, m->n_tets, m->n_nodes, m->n_dof,
                                            f_d, nrhs, b_d);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int load_vector_T(Mesh *m, const double *lam_d, double *out_d) {
    cudaStream_t s = m->stream;
    FEM3_CUDA(cudaMemsetAsync(out_d, 0, sizeof(double) * m->n_nodes, s));
    k_load_T<<<g256(m->n_tets), 256, 0, s>>>(m->tets, m->vol, m->dof, m->n_tets, lam_d, out_d);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// The factorisation is a fixed sequence of ~3 n/64 launches for a given handle and
// precision.  The first factorisation of a handle launches it directly; a second one
// (a new assemble with other alpha or K on the same mesh) captures the sequence into a
// CUDA graph on a private stream, and later ones replay the graph on the caller's stream.
static int chol_attributes() {
    static bool done = false;
    if (done) return FEM3_OK;
    FEM3_CUDA(cudaFuncSetAttribute(k_chol_tiles<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kCholTilesSmem * sizeof(double))));
    FEM3_CUDA(cudaFuncSetAttribute(k_chol_tiles<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(kCholTilesSmem * sizeof(float))));
    done = true;
    return FEM3_OK;
}

// FP32 factorisations of at least this order take the blocked factorisation with
// tensor-core trailing updates (chol_tc.cu); smaller ones the one-launch tile-task
// factorisation, whose diagonal chain is the shorter critical path there.
constexpr int64_t kCholTcMinN = 4096;

int factor(Mesh *m) {
    FEM3_TRY(chol_attributes());
    m->chol_tc_used = false;
    if (m->precision == FEM3_FP64) {
        FEM3_TRY(chol_tiles_t<double>(m->A64, m->n_dof, m->stream, m));
        return solve_prep_t<double>(m->A64, m->n_dof, m->stream, m);
    }
    const bool tc = m->chol_tc_opt > 0 || (m->chol_tc_opt == 0 && m->n_dof >= kCholTcMinN);
    if (tc) {
        FEM3_TRY(chol_tc(m, m->A32, m->n_dof));
        m->chol_tc_used = true;
    } else {
        FEM3_TRY(chol_tiles_t<float>(m->A32, m->n_dof, m->stream, m));
    }
    return solve_prep_t<float>(m->A32, m->n_dof, m->stream, m);
}

// Fused operator apply, one CTA per transverse bin, in double-float arithmetic on the FP32
// pipes.  With R~ = W R (split once per assembly, see k_split_ops), A u restricted to
// the bin is L^T (R~ u) + R~^T (L u) (L read from the table itself).  The bin's Gauss
// points go in chunks of 32, and the chunks are independent: for a chunk, yR = R~ u_b and
// yL = L u_b over its Gauss points (phase 1), then Au += s K (L^T yR + R~^T yL) over the
// chunk's columns (phase 2).  The template rows go in pieces of kApplyRM: a piece's L and
// R~ columns of the chunk are staged in shared memory (cp.async 16-byte copies, zero-filled
// past the bin's Gauss points; rows of 34 pairs, 272 bytes) with u_b as hi + lo pairs and
// the rows' nonzero ranges; phase 2 takes the piece staged last first and stages the others
// again (from L2).
// Rows and Gauss points of a bin are both ordered along the axis, so a row's nonzeros in L
// (paths towards -x) start at a Gauss point that grows with the row and its nonzeros in R~
// end at one: each row carries its exact ranges (k_split_ops) and both phases skip the
// entries outside them, which are exact zeros.
// Phase 1: warp w sums rows w, w + 8, ... (lane = Gauss point, all NR vectors); the eight
// partial sums are added in shared memory.  Phase 2: thread = (row, group of NV vectors) for
// NR = 4 and 8, each over the pairs of Gauss points that hold nonzeros of some row of its
// warp (a warp-uniform range: the yL / yR reads are broadcasts); for NR = 1 thread = (row,
// slice of the pairs), the slices added by shuffles.
// Every product is exact up to 2^-48 relative and sums carry their rounding errors
// (df_fma), so Au matches an FP64 evaluation to a few units in 2^-48.  The kernel has no
// FP64 arithmetic: s K z is formed in double-float FP32 operations and its two parts go to
// Au as exact FP64 values (bit assembly) through FP64 atomics.  NR = 1: u plain; NR = 4, 8:
// u interleaved [dof][NR].
constexpr int kApplyThreads = 256;
constexpr int kApplyGC = 32;                  // Gauss points per chunk
constexpr int kApplyStride = kApplyGC + 2;    // staged row, float2 units: 272 B, 16-B aligned
constexpr int kApplyRM = 64;                  // rows per staged piece

// phase-1 partial-sum buffers: one per warp, or four for NR > 8 (warps 4-7 first add into
// those of warps 0-3)
template <int NR> __host__ __device__ constexpr int apply_pw() { return NR > 8 ? 4 : 8; }
// 76,800 bytes at NR = 8: three CTAs per SM (233,472 bytes less 1,024 reserved per CTA);
// 88,064 bytes at NR = 17: two
template <int NR>
constexpr size_t apply_bin_smem() {
    return (size_t)(2 * kApplyRM * kApplyStride + kApplyRM * NR +
                    2 * apply_pw<NR>() * kApplyGC * NR + 2 * kApplyGC * NR) *
               sizeof(float2) +
           kApplyRM * sizeof(int4);
}

// exact FP64 value of a normal FP32 number (zero and subnormals give 0), by bit assembly:
// exponent rebiased by 1023 - 127, significand moved to the top of the 52-bit field
__device__ __forceinline__ double f32_to_f64_exact(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xFFu;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e + 896u) << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double(e == 0u ? 0ll : (long long)d);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// stage rows [r0, r0 + rn) of the chunk's L and R~ columns [gc0, gc0 + 32): one 16-byte
// copy per (row, pair of Gauss points), the part past the bin's G Gauss points zero-filled
// (and not read: entries past G in a table row are padding); and the rows' nonzero ranges.
// The caller waits (cp.async.wait_all) and synchronises.
__device__ __forceinline__ void apply_stage_ops(const float2 *__restrict__ TL,
                                                const float2 *__restrict__ TR,
                                                const int4 *__restrict__ rng, int ld, int G,
                                                int gc0, int r0, int rn, float2 *Ls,
                                                float2 *Rs, int4 *Qs) {
    for (int e = threadIdx.x; e < rn * 16; e += kApplyThreads) {
        const int r = e >> 4, q = e & 15, g = gc0 + 2 * q;
        const int nb = g + 1 < G ? 16 : (g < G ? 8 : 0);
        const int64_t o = (int64_t)(r0 + r) * ld + (nb ? g : 0);   // in the row when nb = 0
        cp_async16(Ls + r * kApplyStride + 2 * q, TL + o, nb);
        cp_async16(Rs + r * kApplyStride + 2 * q, TR + o, nb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int r = threadIdx.x; r < rn; r += kApplyThreads) Qs[r] = __ldg(rng + r0 + r);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// pairs [p0, p1) of the chunk's Gauss points that hold a row's nonzeros in [first, end)
__device__ __forceinline__ void pair_range(int first, int end, int gc0, int gn, int &p0,
                                           int &p1) {
    p0 = max(first - gc0, 0) >> 1;
    p1 = (min(end - gc0, gn) + 1) >> 1;
}

// phase 2 of one staged piece: thread = (row, group of NV vectors, slice of S of the 16
// pairs of Gauss points); adds s K (L^T yR + R~^T yL) of the chunk to Au
template <int NR, int NV, int S, bool DF>
__device__ __forceinline__ void apply_phase2(const float2 *Ls, const float2 *Rs, const int4 *Qs,
                                             const float2 *yL, const float2 *yR, int rn,
                                             int gc0, int gn, const int32_t *__restrict__ dofs,
                                             float sKh, float sKl, int nv, double *Au,
                                             int64_t ldA) {
    constexpr int VS = NR / NV;   // vector groups per row
    const int t = threadIdx.x;
    const int r = t / (VS * S), vg = (t / S) % VS, s = t % S;   // compile-time divisors
    const bool act = r < rn;
    const int rr = act ? r : 0;
    const int4 q = Qs[rr];
    int l0, l1, q0, q1;
    pair_range(q.x, q.y, gc0, gn, l0, l1);
    pair_range(q.z, q.w, gc0, gn, q0, q1);
    if (!act) { l0 = q0 = kApplyGC; l1 = q1 = 0; }
    if constexpr (S == 1) {
        // the union over the warp's rows (entries outside a row's own range are zeros)
        l0 = __reduce_min_sync(0xffffffffu, l0);
        l1 = __reduce_max_sync(0xffffffffu, l1);
        q0 = __reduce_min_sync(0xffffffffu, q0);
        q1 = __reduce_max_sync(0xffffffffu, q1);
    } else {
        constexpr int PS = (kApplyGC / 2) / S;   // pairs per slice
        l0 = max(l0, s * PS);
        l1 = min(l1, (s + 1) * PS);
        q0 = max(q0, s * PS);
        q1 = min(q1, (s + 1) * PS);
    }
    const float4 *Lr = reinterpret_cast<const float4 *>(Ls + rr * kApplyStride);
    const float4 *Rr = reinterpret_cast<const float4 *>(Rs + rr * kApplyStride);
    const float2 *yRv = yR + vg * NV, *yLv = yL + vg * NV;
    float zh[NV], zl[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) { zh[k] = 0.f; zl[k] = 0.f; }
    for (int g2 = l0; g2 < l1; g2++) {   // two Gauss points per 16-byte read
        const float4 lv = Lr[g2];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const float2 a0 = yRv[2 * g2 * NR + k], a1 = yRv[(2 * g2 + 1) * NR + k];
            if constexpr (DF) {
                df_fma(lv.x, lv.y, a0.x, a0.y, zh[k], zl[k]);
                df_fma(lv.z, lv.w, a1.x, a1.y, zh[k], zl[k]);
            } else {
                zh[k] = fmaf(lv.x, a0.x, zh[k]);
                zh[k] = fmaf(lv.z, a1.x, zh[k]);
            }
        }
    }
    for (int g2 = q0; g2 < q1; g2++) {
        const float4 rv = Rr[g2];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const float2 a0 = yLv[2 * g2 * NR + k], a1 = yLv[(2 * g2 + 1) * NR + k];
            if constexpr (DF) {
                df_fma(rv.x, rv.y, a0.x, a0.y, zh[k], zl[k]);
                df_fma(rv.z, rv.w, a1.x, a1.y, zh[k], zl[k]);
            } else {
                zh[k] = fmaf(rv.x, a0.x, zh[k]);
                zh[k] = fmaf(rv.z, a1.x, zh[k]);
            }
        }
    }
    if constexpr (S > 1) {   // the row's S slices sit in neighbouring lanes
#pragma unroll
        for (int o = 1; o < S; o <<= 1)
#pragma unroll
            for (int k = 0; k < NV; k++) {
                const float xh = __shfl_xor_sync(0xffffffffu, zh[k], o);
                const float xl = __shfl_xor_sync(0xffffffffu, zl[k], o);
                if constexpr (DF) df_add(xh, xl, zh[k], zl[k]);
                else zh[k] += xh;
            }
    }
    // after the butterfly every slice lane holds the row's sums: lane s writes the vectors
    // k = s (mod S)
    if (!act) return;
    const int64_t dof = dofs[r];
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const int v = vg * NV + k;
        if (v >= nv) break;
        if (k % S != s) continue;
        if constexpr (DF) {
            float ph, pl;
            df_mul(zh[k], zl[k], sKh, sKl, ph, pl);
            atomicAdd(&Au[(int64_t)v * ldA + dof], f32_to_f64_exact(ph));
            atomicAdd(&Au[(int64_t)v * ldA + dof], f32_to_f64_exact(pl));
        } else {
            atomicAdd(&Au[(int64_t)v * ldA + dof], (double)(zh[k] * sKh));
        }
    }
}

// one axis of the apply: its bins' operands and s K as an FP32 pair
struct ApplyAxis {
    const float2 *apL, *apR;
    const int4 *rng;   // per template row: Gauss-point ranges of the nonzeros of L and W R
    const int32_t *gp_off, *dof_off, *dof_idx, *tab_ld;
    const int64_t *tab_off;
    float sKh, sKl;
    int n_bins;
};
struct ApplyAxes {
    ApplyAxis a[3];
};

// grid: the bins of the three axes (block x -> axis, bin)
// DF = false: the same operator in plain FP32 arithmetic (hi parts of the table pairs and of
// u, FMA accumulation), about 1e-6 relative: the refinement's late sweeps, whose residual
// update r -= A d has a tiny correction d (see solve_refined)
template <int NR, bool DF = true>
__global__ void __launch_bounds__(kApplyThreads, NR > 8 ? 2 : 3)
    k_apply_bin(const __grid_constant__ ApplyAxes P, const double *__restrict__ u, int nv,
                double *Au, int64_t ldA) {
    static_assert(NR == 1 || NR == 4 || NR == 8 || NR == 17, "vectors per pass");
    constexpr int RM = kApplyRM, PW = apply_pw<NR>();
    int b = blockIdx.x, axis = 0;
    while (axis < 2 && b >= P.a[axis].n_bins) b -= P.a[axis++].n_bins;
    const ApplyAxis &X = P.a[axis];
    const float2 *__restrict__ apL = X.apL, *__restrict__ apR = X.apR;
    const int32_t *__restrict__ gp_off = X.gp_off, *__restrict__ dof_off = X.dof_off,
                  *__restrict__ dof_idx = X.dof_idx, *__restrict__ tab_ld = X.tab_ld;
    const int64_t *__restrict__ tab_off = X.tab_off;
    const float sKh = X.sKh, sKl = X.sKl;
    extern __shared__ __align__(16) float2 sm_apply[];
    float2 *Ls = sm_apply;                       // [RM][34]
    float2 *Rs = Ls + RM * kApplyStride;         // [RM][34]
    float2 *us = Rs + RM * kApplyStride;         // [RM][NR]
    float2 *pL = us + RM * NR;                   // [PW][32][NR] phase-1 partial sums, L u
    float2 *pR = pL + PW * kApplyGC * NR;        // [PW][32][NR] R~ u
    float2 *yL = pR + PW * kApplyGC * NR;        // [32][NR]
    float2 *yR = yL + kApplyGC * NR;             // [32][NR]
    int4 *Qs = reinterpret_cast<int4 *>(yR + kApplyGC * NR);   // [RM] row ranges
    const int d0 = dof_off[b], D = dof_off[b + 1] - d0;
    const int G = gp_off[b + 1] - gp_off[b], ld = tab_ld[b];
    if (D == 0 || G == 0) return;
    const float2 *TL = apL + tab_off[b], *TR = apR + tab_off[b];
    const int4 *rng = X.rng + d0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int np = (D + RM - 1) / RM;
    for (int gc0 = 0; gc0 < G; gc0 += kApplyGC) {
        const int gn = min(kApplyGC, G - gc0);
        // ---- phase 1: lane = Gauss point gc0 + lane, warp = row slice ----
        float lh[NR], ll[NR], rh[NR], rl[NR];
#pragma unroll
        for (int v = 0; v < NR; v++) { lh[v] = 0.f; ll[v] = 0.f; rh[v] = 0.f; rl[v] = 0.f; }
        for (int p = 0; p < np; p++) {
            const int rc0 = p * RM, rn = min(RM, D - rc0);
            __syncthreads();   // earlier readers of the staged rows are done
            apply_stage_ops(TL, TR, rng, ld, G, gc0, rc0, rn, Ls, Rs, Qs);
            for (int e = tid; e < rn * NR; e += kApplyThreads) {
                const int r = e / NR, v = e - r * NR;
                const int64_t dof = dof_idx[d0 + rc0 + r];
                float a, a2;
                f64_split(NR == 1 ? u[dof] : u[dof * NR + v], a, a2);
                us[e] = make_float2(a, a2);
            }
            cp_async_wait_all();
            __syncthreads();
            for (int r = warp; r < rn; r += kApplyThreads / 32) {
                // does the row's nonzero range meet this chunk in L, in R~?  (usually one)
                const int4 q = Qs[r];
                if (q.x < gc0 + kApplyGC && q.y > gc0) {
                    const float2 lv = Ls[r * kApplyStride + lane];
#pragma unroll
                    for (int v = 0; v < NR; v++) {
                        const float2 uv = us[r * NR + v];
                        if constexpr (DF) df_fma(lv.x, lv.y, uv.x, uv.y, lh[v], ll[v]);
                        else lh[v] = fmaf(lv.x, uv.x, lh[v]);
                    }
                }
                if (q.z < gc0 + kApplyGC && q.w > gc0) {
                    const float2 rv = Rs[r * kApplyStride + lane];
#pragma unroll
                    for (int v = 0; v < NR; v++) {
                        const float2 uv = us[r * NR + v];
                        if constexpr (DF) df_fma(rv.x, rv.y, uv.x, uv.y, rh[v], rl[v]);
                        else rh[v] = fmaf(rv.x, uv.x, rh[v]);
                    }
                }
            }
        }
        if constexpr (PW == 8) {
#pragma unroll
            for (int v = 0; v < NR; v++) {
                pL[(warp * kApplyGC + lane) * NR + v] = make_float2(lh[v], ll[v]);
                pR[(warp * kApplyGC + lane) * NR + v] = make_float2(rh[v], rl[v]);
            }
        } else {
            // warps 4-7 store, warps 0-3 add their own sums to them
            const int w4 = warp & 3;
            if (warp >= 4) {
#pragma unroll
                for (int v = 0; v < NR; v++) {
                    pL[(w4 * kApplyGC + lane) * NR + v] = make_float2(lh[v], ll[v]);
                    pR[(w4 * kApplyGC + lane) * NR + v] = make_float2(rh[v], rl[v]);
                }
            }
            __syncthreads();
            if (warp < 4) {
#pragma unroll
                for (int v = 0; v < NR; v++) {
                    const int e = (w4 * kApplyGC + lane) * NR + v;
                    const float2 x = pL[e], z = pR[e];
                    if constexpr (DF) {
                        df_add(x.x, x.y, lh[v], ll[v]);
                        df_add(z.x, z.y, rh[v], rl[v]);
                    } else {
                        lh[v] += x.x;
                        rh[v] += z.x;
                    }
                    pL[e] = make_float2(lh[v], ll[v]);
                    pR[e] = make_float2(rh[v], rl[v]);
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < kApplyGC * NR; e += kApplyThreads) {
            float2 a = pL[e], c = pR[e];
            float ah = a.x, al = a.y, ch = c.x, cl = c.y;
#pragma unroll
            for (int w = 1; w < PW; w++) {
                const float2 x = pL[w * kApplyGC * NR + e], z = pR[w * kApplyGC * NR + e];
                if constexpr (DF) {
                    df_add(x.x, x.y, ah, al);
                    df_add(z.x, z.y, ch, cl);
                } else {
                    ah += x.x;
                    ch += z.x;
                }
            }
            yL[e] = make_float2(ah, al);
            yR[e] = make_float2(ch, cl);
        }
        __syncthreads();
        // ---- phase 2: the piece staged last first ----
        for (int pass = 0; pass < np; pass++) {
            const int p = pass == 0 ? np - 1 : pass - 1;
            const int rc0 = p * RM, rn = min(RM, D - rc0);
            if (pass > 0) {
                __syncthreads();
                apply_stage_ops(TL, TR, rng, ld, G, gc0, rc0, rn, Ls, Rs, Qs);
                cp_async_wait_all();
                __syncthreads();
            }
            const int32_t *dofs = dof_idx + d0 + rc0;
            if constexpr (NR == 8) {
                if (rn <= 32)
                    apply_phase2<8, 1, 1, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
                else
                    apply_phase2<8, 2, 1, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
            } else if constexpr (NR == 4) {
                if (rn <= 32)
                    apply_phase2<4, 1, 2, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
                else
                    apply_phase2<4, 1, 1, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
            } else if constexpr (NR == 17) {
                if (rn <= 32)
                    apply_phase2<17, 17, 8, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl,
                                                nv, Au, ldA);
                else
                    apply_phase2<17, 17, 4, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl,
                                                nv, Au, ldA);
            } else {
                if (rn <= 32)
                    apply_phase2<1, 1, 8, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
                else
                    apply_phase2<1, 1, 4, DF>(Ls, Rs, Qs, yL, yR, rn, gc0, gn, dofs, sKh, sKl, nv,
                                              Au, ldA);
            }
        }
    }
}

// The same operator from the lists of the tables' nonzeros (the Gauss-point-major and
// row-major lists that k_gp_lists and k_split_ops write with the apply operands): the work is
// the nonzeros, about a fifth of the dense bin blocks (a Gauss point's line crosses the
// element patches of a few of its bin's template dofs).  One CTA per bin, one y buffer:
//   phase 0: u of the bin's template rows into shared memory (hi + lo pairs, [D][NR]);
//   then two rounds, (point table, row table) = (W R, L) and then (L, W R):
//   phase 1, warp = (chunk of 32 Gauss points, half of the vectors), lane = point: y[g] =
//     sum over g's list in the point table of T[r][g] u[r], into shared memory ([G][NR]; the
//     chunk layout puts the lanes' entries k side by side);
//   phase 2, thread = up to two items (template row r, group of NV vectors): z += sum over
//     r's list in the row table of T'[r][g] y[g], z kept in registers across the rounds;
//   at the end Au[dof(r)] += s K z (FP64 atomics of the double-float parts, as in
//   k_apply_bin).
// With rows and Gauss points ordered along the axis, a point's L list grows along the bin as
// its W R list shrinks (and likewise for a row), so the lanes of a warp do similar work.
// u comes split into hi + lo FP32 pairs, [dof][NR] (k_split_vec).  The bin's rows, Gauss
// points and their NR sums must fit the launch's shared memory (apply_multi checks).
template <int NR>
__global__ void k_split_vec(const double *__restrict__ u, int64_t n, int nv, float2 *uf) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NR * n) return;
    const int64_t i = e / NR;
    const int v = (int)(e - i * NR);
    float h = 0.f, l = 0.f;
    if (v < nv) f64_split(u[(int64_t)v * n + i], h, l);
    uf[e] = make_float2(h, l);
}

// loads that do not happen when `pred` is false (a predicated PTX load: no access is made, the
// address need not be valid, and the result keeps its zero)
__device__ __forceinline__ float2 ldg_if(const float2 *p, bool pred) {
    float x = 0.f, y = 0.f;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t"
        "@q ld.global.nc.v2.f32 {%0, %1}, [%3];\n\t}"
        : "+f"(x), "+f"(y)
        : "r"((int)pred), "l"(p));
    return make_float2(x, y);
}
__device__ __forceinline__ int ldg_if(const uint16_t *p, bool pred) {
    uint32_t v = 0;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t"
        "@q ld.global.nc.u16 %0, [%2];\n\t}"
        : "+r"(v)
        : "r"((int)pred), "l"(p));
    return (int)v;
}

struct ListAxis {
    const uint16_t *rg[2];          // row-major lists: Gauss-point index, value (t = 0 L, 1 W R)
    const float2 *rv[2];
    const int32_t *rn[2];
    const uint16_t *gr[2];          // Gauss-point-major lists (chunk layout): row index, value
    const float2 *gv[2];
    const int32_t *gn[2];
    const int32_t *gp_off, *dof_off, *dof_idx, *tab_ld;
    const int64_t *tab_off;
    float sKh, sKl;
    int n_bins;
};
struct ListAxes {
    ListAxis a[3];
};

constexpr int kListThreads = 256;
constexpr int kListBatch = 3;   // list entries whose loads are in flight together (timed: 3 of 2, 3, 4)

template <int NR, int VS, bool DF>
__global__ void __launch_bounds__(kListThreads, 3) k_apply_lists(const __grid_constant__ ListAxes P,
                                                              const float2 *__restrict__ uf,
                                                              int nv, double *Au, int64_t ldA,
                                                              int max_dof) {
    constexpr int NV = (NR + VS - 1) / VS;   // phase-2 vectors per item (the last group short)
    constexpr int NH = (NR + 1) / 2;         // phase-1 vectors per warp item (two halves)
    int b = blockIdx.x, axis = 0;
    while (axis < 2 && b >= P.a[axis].n_bins) b -= P.a[axis++].n_bins;
    const ListAxis &X = P.a[axis];
    const int d0 = X.dof_off[b], D = X.dof_off[b + 1] - d0;
    const int g0 = X.gp_off[b], G = X.gp_off[b + 1] - g0;
    if (D == 0 || G == 0) return;
    const int ld = X.tab_ld[b];
    const int64_t t0 = X.tab_off[b];
    extern __shared__ __align__(16) float2 sm_lists[];
    float2 *us = sm_lists;                         // [max_dof][NR]
    float2 *y = us + (int64_t)max_dof * NR;        // [G][NR]: R~ u, then L u
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // phase-2 items (row, vector group) of this thread, fixed for both rounds
    float zh[kListItems][NV], zl[kListItems][NV];
#pragma unroll
    for (int i = 0; i < kListItems; i++)
#pragma unroll
        for (int k = 0; k < NV; k++) { zh[i][k] = 0.f; zl[i][k] = 0.f; }
    // ---- phase 0 ----
    for (int e = tid; e < D * NR; e += kListThreads) {
        const int c = e / NR, v = e - c * NR;
        us[e] = __ldg(uf + (int64_t)__ldg(X.dof_idx + d0 + c) * NR + v);
    }
    // Round 0: y = R~ u from the points' W R lists, then the rows' L lists against it;
    // round 1: y = L u from the points' L lists, then the rows' W R lists.
#pragma unroll
    for (int round = 0; round < 2; round++) {
        const int tg = 1 - round, tr = round;   // point-list table, row-list table
        __syncthreads();   // u staged / the rows are done with the previous round's y
        // ---- phase 1: warp = (chunk of 32 Gauss points, half of the vectors), lane = point
        const int nchunk = (G + 31) >> 5;
        for (int wi = warp; wi < 2 * nchunk; wi += kListThreads / 32) {
            const int gc = 32 * (wi >> 1), v0 = NH * (wi & 1);
            const int g = gc + lane, wc = min(32, G - gc);
            const bool in = g < G;
            const int64_t base = t0 + (int64_t)gc * D + lane;
            float h[NH], l[NH];
#pragma unroll
            for (int k = 0; k < NH; k++) { h[k] = 0.f; l[k] = 0.f; }
            const int cnt = in ? X.gn[tg][g0 + g] : 0;
            const int cmax = __reduce_max_sync(0xffffffffu, cnt);
            const uint16_t *__restrict__ rl = X.gr[tg] + base;
            const float2 *__restrict__ vl = X.gv[tg] + base;
            for (int q0 = 0; q0 < cmax; q0 += kListBatch) {
                float2 a[kListBatch];
                int r[kListBatch];
#pragma unroll
                for (int j = 0; j < kListBatch; j++) {
                    // only the lane's own entries are read (cnt = 0 past the bin's points)
                    const bool ok = q0 + j < cnt;
                    const int64_t o = (int64_t)(q0 + j) * wc;
                    a[j] = ldg_if(vl + o, ok);
                    r[j] = ldg_if(rl + o, ok);
                }
#pragma unroll
                for (int j = 0; j < kListBatch; j++) {
                    const float2 *ur = us + r[j] * NR + v0;
#pragma unroll
                    for (int k = 0; k < NH; k++) {
                        if (v0 + k >= NR) break;
                        const float2 uu = ur[k];
                        if constexpr (DF) df_fma(a[j].x, a[j].y, uu.x, uu.y, h[k], l[k]);
                        else h[k] = fmaf(a[j].x, uu.x, h[k]);
                    }
                }
            }
            if (in) {
                float2 *yg = y + (int64_t)g * NR + v0;
#pragma unroll
                for (int k = 0; k < NH; k++)
                    if (v0 + k < NR) yg[k] = make_float2(h[k], l[k]);
            }
        }
        __syncthreads();
        // ---- phase 2: the thread's rows, their table-tr lists against y ----
#pragma unroll
        for (int i = 0; i < kListItems; i++) {
            const int it = tid + i * kListThreads;
            if (it >= D * VS) break;
            const int c = it / VS, v0 = (it - c * VS) * NV;
            const int64_t base = t0 + (int64_t)c * ld;
            const int cnt = X.rn[tr][d0 + c];
            const uint16_t *__restrict__ gl = X.rg[tr] + base;
            const float2 *__restrict__ vl = X.rv[tr] + base;
            for (int q0 = 0; q0 < cnt; q0 += kListBatch) {
                float2 a[kListBatch];
                int gi[kListBatch];
#pragma unroll
                for (int j = 0; j < kListBatch; j++) {
                    // the row's own entries only
                    const bool ok = q0 + j < cnt;
                    a[j] = ldg_if(vl + q0 + j, ok);
                    gi[j] = ldg_if(gl + q0 + j, ok);
                }
#pragma unroll
                for (int j = 0; j < kListBatch; j++) {
                    const float2 *yr = y + gi[j] * NR + v0;
#pragma unroll
                    for (int k = 0; k < NV; k++) {
                        if (v0 + k >= NR) break;
                        const float2 yy = yr[k];
                        if constexpr (DF) df_fma(a[j].x, a[j].y, yy.x, yy.y, zh[i][k], zl[i][k]);
                        else zh[i][k] = fmaf(a[j].x, yy.x, zh[i][k]);
                    }
                }
            }
        }
    }
    // ---- the thread's rows into Au ----
#pragma unroll
    for (int i = 0; i < kListItems; i++) {
        const int it = tid + i * kListThreads;
        if (it >= D * VS) break;
        const int c = it / VS, v0 = (it - c * VS) * NV;
        const int64_t dof = X.dof_idx[d0 + c];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            const int v = v0 + k;
            if (v >= NR || v >= nv) break;
            if constexpr (DF) {
                float ph, pl;
                df_mul(zh[i][k], zl[i][k], X.sKh, X.sKl, ph, pl);
                atomicAdd(&Au[(int64_t)v * ldA + dof], f32_to_f64_exact(ph));
                atomicAdd(&Au[(int64_t)v * ldA + dof], f32_to_f64_exact(pl));
            } else {
                atomicAdd(&Au[(int64_t)v * ldA + dof], (double)(zh[i][k] * X.sKh));
            }
        }
    }
}

// Au = A u for nv vectors (column-major, leading dimension n_dof), applied from
// the tables; vectors go through the tables in groups: up to 17 per pass while at least 13
// are left, then up to eight, and a last group of one or up to four vectors takes the
// narrower form of the kernel (a pass costs a fixed part, staging and the phases' overhead,
// plus about its vectors' arithmetic: an eight-wide pass for one leftover vector cost as much
// as a full group).
int apply_multi(Mesh *m, const double *u_d, int nv, double *Au_d, bool df) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    FEM3_CUDA(cudaMemsetAsync(Au_d, 0, sizeof(double) * n * nv, s));
    static bool attr = false;
    if (!attr) {
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<1>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<4>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<8>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<1, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<1>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<4, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<4>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<8, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<8>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<17>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<17>()));
        FEM3_CUDA(cudaFuncSetAttribute(k_apply_bin<17, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)apply_bin_smem<17>()));
        attr = true;
    }
    FEM3_TRY(ap_prepare(m));
    ApplyAxes P;
    ListAxes PL;
    int64_t nblk = 0;
    int max_gp = 0, max_dof = 0;
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        const bool on = B.n_tmpl > 0 && B.n_bins > 0;
        const float skh = (float)m->sK[axis], skl = (float)(m->sK[axis] - (double)skh);
        P.a[axis] = ApplyAxis{m->tabL[axis], B.ap_R, B.ap_rng, B.gp_off, B.dof_off, B.dof_idx,
                              B.tab_ld, B.tab_off, skh, skl, on ? B.n_bins : 0};
        PL.a[axis] = ListAxis{{B.rl_g[0], B.rl_g[1]}, {B.rl_v[0], B.rl_v[1]},
                              {B.rl_n[0], B.rl_n[1]}, {B.gl_r[0], B.gl_r[1]},
                              {B.gl_v[0], B.gl_v[1]}, {B.gl_n[0], B.gl_n[1]},
                              B.gp_off, B.dof_off, B.dof_idx, B.tab_ld, B.tab_off, skh, skl,
                              on ? B.n_bins : 0};
        nblk += on ? B.n_bins : 0;
        if (on) {
            max_gp = std::max(max_gp, B.max_gp);
            max_dof = std::max(max_dof, B.max_dof);
        }
    }
    // the lists' kernel when the largest bin's Gauss points and their 17 sums fit
    const bool lists = apply_lists_fit(m);
    if (lists) {
        static bool lattr = false;
        if (!lattr) {
#define FEM3_LATTR(NR_, VS_)                                                                     \
    FEM3_CUDA(cudaFuncSetAttribute(k_apply_lists<NR_, VS_, true>,                                \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kListSmemMax)); \
    FEM3_CUDA(cudaFuncSetAttribute(k_apply_lists<NR_, VS_, false>,                               \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kListSmemMax))
            FEM3_LATTR(17, 2);
            FEM3_LATTR(8, 2);
            FEM3_LATTR(4, 2);
            FEM3_LATTR(1, 1);
#undef FEM3_LATTR
            lattr = true;
        }
    }
    double *ui = nullptr;
    if (nv > 1 || lists)
        FEM3_CUDA(cudaMallocAsync((void **)&ui, sizeof(double) * 17 * std::max<int64_t>(1, n), s));
    float2 *uf = reinterpret_cast<float2 *>(ui);
    for (int v0 = 0, cnt = 0; v0 < nv && nblk > 0; v0 += cnt) {
        const int left = nv - v0;
        const int nri = left >= 13 ? 17 : (left >= 5 ? 8 : (left >= 2 ? 4 : 1));
        cnt = std::min(nri, left);
        double *out = Au_d + (int64_t)v0 * n;
        if (lists) {
            const double *us = u_d + (int64_t)v0 * n;
            const size_t sh = apply_lists_smem(nri, max_dof, max_gp);
#define FEM3_LISTS(NR_, VS_)                                                                     \
    do {                                                                                         \
        k_split_vec<NR_><<<g256((int64_t)NR_ * n), 256, 0, s>>>(us, n, cnt, uf);                 \
        note_launch(m);                                                                          \
        kc_begin(m, KC_APPLY);                                                                   \
        if (df)                                                                                  \
            k_apply_lists<NR_, VS_, true><<<(unsigned)nblk, kListThreads, sh, s>>>(PL, uf, cnt,  \
                                                                                 out, n, max_dof); \
        else                                                                                     \
            k_apply_lists<NR_, VS_, false><<<(unsigned)nblk, kListThreads, sh, s>>>(PL, uf, cnt, \
                                                                                  out, n, max_dof); \
        kc_end(m, KC_APPLY);                                                                     \
        note_launch(m);                                                                          \
    } while (0)
            if (nri == 17) FEM3_LISTS(17, 2);
            else if (nri == 8) FEM3_LISTS(8, 2);
            else if (nri == 4) FEM3_LISTS(4, 2);
            else FEM3_LISTS(1, 1);
#undef FEM3_LISTS
            continue;
        }
        if (nri == 4)
            k_interleave<4><<<g256(4 * n), 256, 0, s>>>(u_d + (int64_t)v0 * n, n, cnt, ui);
        else if (nri == 8)
            k_interleave<8><<<g256(8 * n), 256, 0, s>>>(u_d + (int64_t)v0 * n, n, cnt, ui);
        else if (nri == 17)
            k_interleave<17><<<g256(17 * n), 256, 0, s>>>(u_d + (int64_t)v0 * n, n, cnt, ui);
        if (nri > 1) note_launch(m);
        kc_begin(m, KC_APPLY);
#define FEM3_APPLY(NR_, DF_, U_, CNT_)                                                          \
    k_apply_bin<NR_, DF_><<<(unsigned)nblk, kApplyThreads, apply_bin_smem<NR_>(), s>>>(P, U_, CNT_, \
                                                                                   out, n)
        if (nri == 1) {
            if (df) FEM3_APPLY(1, true, u_d + (int64_t)v0 * n, 1);
            else FEM3_APPLY(1, false, u_d + (int64_t)v0 * n, 1);
        } else if (nri == 4) {
            if (df) FEM3_APPLY(4, true, ui, cnt);
            else FEM3_APPLY(4, false, ui, cnt);
        } else if (nri == 8) {
            if (df) FEM3_APPLY(8, true, ui, cnt);
            else FEM3_APPLY(8, false, ui, cnt);
        } else {
            if (df) FEM3_APPLY(17, true, ui, cnt);
            else FEM3_APPLY(17, false, ui, cnt);
        }
#undef FEM3_APPLY
        kc_end(m, KC_APPLY);
        note_launch(m);
    }
    if (ui) FEM3_CUDA(cudaFreeAsync(ui, s));
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int apply_A64(Mesh *m, const double *u_d, double *Au_d) { return apply_multi(m, u_d, 1, Au_d, true); }

int axis_forms(Mesh *m, const double *u_d, const double *lam_d, double out[3]) {
    cudaStream_t s = m->stream;
    FEM3_CUDA(cudaFuncSetAttribute(k_axis_form, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(double) * 2 * kMaxBinItems)));
    FEM3_CUDA(cudaMemsetAsync(m->norms, 0, sizeof(double) * 3, s));
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        size_t sh = sizeof(double) * 2 * B.max_dof;
        k_axis_form<<<B.n_bins, 256, sh, s>>>(m->tabL[axis], m->tabR[axis], B.gp_off, B.gp_idx,
                                               B.dof_off, B.dof_idx, B.tab_off, B.tab_ld, m->gw, u_d,
                                               lam_d, m->norms + axis);
        note_launch(m);
    }
    FEM3_CUDA(cudaMemcpyAsync(m->h_norms, m->norms, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    for (int a = 0; a < 3; a++) out[a] = m->s[a] * m->h_norms[a];
    return FEM3_OK;
}

int solve_direct(Mesh *m, const double *b_d, int nrhs, double *u_d) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    FEM3_CUDA(cudaMemcpyAsync(u_d, b_d, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, s));
    for (int c0 = 0; c0 < nrhs; c0 += kMaxRhs)
        FEM3_TRY(trsm_t<double>(m->A64, n, u_d + (int64_t)c0 * n, std::min(kMaxRhs, nrhs - c0), s, m));
    return FEM3_OK;
}

// Refinement for all right-hand sides together: u = 0, r = b; repeat
//   d = A32^{-1} r (FP32 factor, all columns in one wavefront sweep pair), u += d,
//   r = b - A u (FP64 operator from the tables, double-float arithmetic),
// until every column has ||r|| <= tol ||b|| or max_iter sweeps.  Once the residual is below
// kLateFactor * tol, a sweep's residual is updated from its correction alone,
// r = r - A d, with A d applied in plain FP32 (about 1e-6 relative): d is as small as r, so
// the update's error is about 1e-6 ||r|| <= 1e-6 kLateFactor tol ||b|| = tol ||b|| / 100,
// while the double-float apply of A u costs six times the instructions.
constexpr double kLateFactor = 1e4;

int solve_refined(Mesh *m, const double *b_d, int nrhs, double tol, int max_iter, double *u_d,
                  int *iters, double *resid) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    const int64_t nn = n * nrhs;
    if (nrhs > 32) return set_error(FEM3_E_ARG, "at most 32 right-hand sides per solve");
    double *Au = nullptr, *r = nullptr, *d64 = nullptr;
    float *r32 = nullptr;
    FEM3_CUDA(cudaMallocAsync((void **)&Au, sizeof(double) * nn, s));
    FEM3_CUDA(cudaMallocAsync((void **)&r, sizeof(double) * nn, s));
    FEM3_CUDA(cudaMallocAsync((void **)&d64, sizeof(double) * nn, s));
    FEM3_CUDA(cudaMallocAsync((void **)&r32, sizeof(float) * nn, s));
    FEM3_CUDA(cudaMemsetAsync(u_d, 0, sizeof(double) * nn, s));
    FEM3_CUDA(cudaMemcpyAsync(r, b_d, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
    int it = 0;
    double worst = 1.0;
    bool late = false;
    int st = FEM3_OK;
    for (;;) {
        k_to_f32<<<g256(nn), 256, 0, s>>>(r, r32, nn);
        note_launch(m);
        for (int c0 = 0; c0 < nrhs && st == FEM3_OK; c0 += kMaxRhs)
            st = trsm_t<float>(m->A32, n, r32 + c0 * n, std::min(kMaxRhs, nrhs - c0), s, m);
        if (st != FEM3_OK) break;
        k_axpy_f32<<<g256(nn), 256, 0, s>>>(r32, u_d, nn);
        note_launch(m);
        FEM3_CUDA(cudaMemsetAsync(m->norms, 0, sizeof(double) * 2 * nrhs, s));
        if (late) {
            k_f32_to_f64_n<<<g256(nn), 256, 0, s>>>(r32, d64, nn);
            note_launch(m);
            if ((st = apply_multi(m, d64, nrhs, Au, false)) != FEM3_OK) break;
            k_residual_update_cols<<<dim3(g256(n), nrhs), 256, 0, s>>>(b_d, Au, n, r, m->norms);
        } else {
            if ((st = apply_multi(m, u_d, nrhs, Au, true)) != FEM3_OK) break;
            k_residual_cols<<<dim3(g256(n), nrhs), 256, 0, s>>>(b_d, Au, n, r, m->norms);
        }
        note_launch(m);
        FEM3_CUDA(cudaMemcpyAsync(m->h_norms, m->norms, sizeof(double) * 2 * nrhs,
                                  cudaMemcpyDeviceToHost, s));
        FEM3_CUDA(cudaStreamSynchronize(s));
        worst = 0;
        for (int c = 0; c < nrhs; c++) {
            const double rel = m->h_norms[2 * c + 1] > 0 ? sqrt(m->h_norms[2 * c] / m->h_norms[2 * c + 1]) : 0.0;
            worst = (rel == rel) ? std::max(worst, rel) : INFINITY;
        }
        it++;
        if (worst <= tol || it >= max_iter || !(worst < INFINITY)) break;
        late = worst <= kLateFactor * tol;
    }
    cudaFreeAsync(d64, s);
    cudaFreeAsync(Au, s);
    cudaFreeAsync(r, s);
    cudaFreeAsync(r32, s);
    if (iters) *iters = it;
    if (resid) *resid = worst;
    if (st != FEM3_OK) return st;
    if (!(worst <= tol))
        return set_error(FEM3_E_NO_CONVERGE, "iterative refinement did not reach the tolerance");
    return FEM3_OK;
}

}  // namespace fem3
