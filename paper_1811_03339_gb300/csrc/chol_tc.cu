// Blocked right-looking Cholesky A = L L^T in FP32 with the trailing updates on the tensor
// cores (tcgen05, TF32 x 3 split products, FP32 accumulation), for the mixed forms' large
// matrices.  The factor is used as the preconditioner of the FP64 iterative refinement
// (the mixed forms' solve), so it needs the accuracy of an FP32 factorisation, which the
// split products keep (about 2^-21 relative per product against 2^-10 for one TF32
// product).
//
// Per panel of P = 128 columns [j0, j0 + P):
//   1. k_cholp_diag (one CTA): the 128 x 128 diagonal block as two 64 x 64 blocks - factor
//      and invert D11 (X11 = L11^{-1}), L21 = A21 X11^T, factor and invert D22 - L21 L21^T;
//      X11 and X22 go to dinv and L21 to A, the layout the triangular-solve chains read (the
//      strictly lower 64 x 64 tiles of A hold L; a diagonal tile is only used through its
//      inverse), and [X11 | X22 | L21] to the panel solve;
//   2. k_cholp_panel: for every row below the panel, L[:, 0:64] = A[:, 0:64] X11^T and
//      L[:, 64:128] = (A[:, 64:128] - L[:, 0:64] L21^T) X22^T, into A and, split into TF32
//      hi + lo pairs, into the K-major operand rows W_hi, W_lo;
//   3. k_cholp_trail (persistent): A[I, J] -= W_I W_J^T over the 128 x 128 tiles I >= J of
//      the trailing matrix - TMA loads (128-byte swizzle) into a two-stage ring, three MMAs
//      per 32-column K step (hi hi, hi lo, lo hi) into one of two TMEM accumulators, and an
//      epilogue (sixteen warps) that overlaps the next tile's MMAs.
// Look-ahead: the next panel's block column is updated on the caller's stream and the rest of
// the trailing matrix on a side stream, so the next diagonal block and panel overlap it.
// No kernel waits for another CTA; the mbarrier waits are bounded (ERR_CHOL on expiry).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

#include "chol_smem.cuh"

constexpr int kWaitLimit = 1 << 22;
#include "tc_ptx.cuh"

constexpr int kP = 128;                        // panel width
constexpr int kLd = NB + 1;                    // shared 64 x 64 block row stride
constexpr int kDiagSmemFloats = 6 * NB * kLd;  // a_s, x_s, b_s (A21 -> L21), x11, t, A22
constexpr int kPanelRows = 64;                 // rows of a panel-solve CTA
constexpr uint32_t kTile = 128 * 128;          // bytes of one 128-row x 128-byte TMA box
constexpr uint32_t kStage = 4 * kTile;         // A hi, A lo, B hi, B lo: 64 KB
constexpr int kStages = 2;
constexpr int kCsLd = 129;                     // row stride of the staged C tile (floats)
constexpr uint32_t kCsBytes = 128 * kCsLd * 4;  // 66 KB
constexpr uint32_t kTrailSmem = kStages * kStage + kCsBytes + 1024 + 256;
constexpr int kTrailThreads = 576;              // TMA warp, MMA warp, sixteen epilogue warps
constexpr int kEpiThreads = 512;
constexpr int kReservedSms = 20;                // left to the critical chain by the bulk update

// ------------------------------- diagonal block ----------------------------------
// c[i][j] (+)= sgn * sum_k a[i][k] b(k, j) over a 64 x 64 x 64 product in shared memory,
// 512 threads, 8 outputs each; BT selects b(k, j) = b[j][k] (transposed) or b[k][j].
template <bool BT>
__device__ __forceinline__ void smem_gemm64(float (*c)[kLd], const float (*a)[kLd],
                                            const float (*b)[kLd], float sgn, bool accumulate) {
    const int tid = threadIdx.x, r = tid >> 3, c0 = (tid & 7) * 8;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = 0.f;
    for (int k = 0; k < NB; k++) {
        const float av = a[r][k];
#pragma unroll
        for (int q = 0; q < 8; q++) acc[q] = fmaf(av, BT ? b[c0 + q][k] : b[k][c0 + q], acc[q]);
    }
    __syncthreads();   // c may alias an operand's storage in the caller's sequence
#pragma unroll
    for (int q = 0; q < 8; q++) c[r][c0 + q] = (accumulate ? c[r][c0 + q] : 0.f) + sgn * acc[q];
    __syncthreads();
}

// one CTA of 512 threads: the diagonal block [j0, j0 + nbp) of A (nbp <= 128).  Every global
// load of the block is issued first; then D11 = L11 L11^T with X11 = L11^{-1}, L21 = A21 X11^T,
// D22 - L21 L21^T = L22 L22^T with X22 = L22^{-1}.  Out: X11, X22 into dinv (the
// triangular-solve chains' diagonal inverses), L21 into A, and [X11 | X22 | L21] (three
// 64 x 64 blocks, row-major) into Pinv for the panel solve.
__global__ void __launch_bounds__(512, 1) k_cholp_diag(float *A, int64_t n, int64_t j0, int nbp,
                                                       float *dinv, float *Pinv, int32_t *err) {
    extern __shared__ __align__(16) float sm_diag[];
    float(*a_s)[kLd] = reinterpret_cast<float(*)[kLd]>(sm_diag);
    float(*x_s)[kLd] = a_s + NB;
    float(*b_s)[kLd] = x_s + NB;   // A21, then L21
    float(*x11)[kLd] = b_s + NB;
    float(*t_s)[kLd] = x11 + NB;   // L21 L21^T
    float(*d22)[kLd] = t_s + NB;   // A22 as loaded
    const int tid = threadIdx.x;
    const int nb1 = min(NB, nbp), nb2 = nbp - nb1;
    for (int e = tid; e < NB * NB; e += 512) {
        const int i = e >> 6, c = e & 63;
        a_s[i][c] = (i < nb1 && c < nb1) ? A[(j0 + i) * n + j0 + c] : (i == c ? 1.f : 0.f);
        b_s[i][c] = (i < nb2) ? A[(j0 + NB + i) * n + j0 + c] : 0.f;
        d22[i][c] = (i < nb2 && c < nb2) ? A[(j0 + NB + i) * n + j0 + NB + c] : (i == c ? 1.f : 0.f);
    }
    __syncthreads();
    potrf_inv_smem<float>(a_s, x_s, nb1, j0, err);
    float *d1 = dinv + (j0 / NB) * (int64_t)NB * NB;
    for (int e = tid; e < NB * NB; e += 512) {
        const int i = e >> 6, c = e & 63;
        d1[e] = x_s[i][c];
        x11[i][c] = x_s[i][c];
        Pinv[e] = x_s[i][c];
    }
    if (nb2 > 0) {
        __syncthreads();
        smem_gemm64<true>(b_s, b_s, x11, 1.f, false);          // b_s = L21 = A21 X11^T
        smem_gemm64<true>(t_s, b_s, b_s, 1.f, false);          // t = L21 L21^T
        for (int e = tid; e < NB * NB; e += 512) {
            const int i = e >> 6, c = e & 63;
            if (i < nb2) A[(j0 + NB + i) * n + j0 + c] = b_s[i][c];
            Pinv[2 * NB * NB + e] = b_s[i][c];
            // the identity padding stays: L21's padded rows are zero
            a_s[i][c] = d22[i][c] - t_s[i][c];
        }
        __syncthreads();
        potrf_inv_smem<float>(a_s, x_s, nb2, j0 + NB, err);    // x_s = X22
        float *d2 = d1 + (int64_t)NB * NB;
        for (int e = tid; e < NB * NB; e += 512) {
            d2[e] = x_s[e >> 6][e & 63];
            Pinv[NB * NB + e] = x_s[e >> 6][e & 63];
        }
    }
}

// ------------------------------- panel solve --------------------------------------
// rows [r0, r0 + 64) below the panel (r0 >= t0 = j0 + P), in two 64-column steps:
//   L[:, 0:64]   = A[:, 0:64] X11^T
//   L[:, 64:128] = (A[:, 64:128] - L[:, 0:64] L21^T) X22^T
// written to A and, as TF32 hi + lo, to the operand rows W[i - t0] of the trailing update.
// 256 threads, each 4 rows x 4 columns of every 64 x 64 product.
constexpr int kQ = 68;   // shared row stride (floats) of the 64-wide blocks: 16-byte rows
__device__ __forceinline__ void panel_gemm64(const float (*a)[kQ], const float (*bt)[kQ],
                                             float acc[4][4], int ty, int tx) {
    // acc[p][q] += sum_k a[4 ty + p][k] bt[k][4 tx + q]
#pragma unroll 4
    for (int k = 0; k < 64; k++) {
        const float4 b4 = *reinterpret_cast<const float4 *>(&bt[k][4 * tx]);
        const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int p = 0; p < 4; p++) {
            const float av = a[4 * ty + p][k];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[p][q] = fmaf(av, bv[q], acc[p][q]);
        }
    }
}

__global__ void __launch_bounds__(256) k_cholp_panel(float *A, int64_t n, int64_t j0,
                                                     const float *__restrict__ Pinv, float *Whi,
                                                     float *Wlo) {
    extern __shared__ __align__(16) float sm_panel[];
    float(*x11t)[kQ] = reinterpret_cast<float(*)[kQ]>(sm_panel);   // x11t[k][c] = X11[c][k]
    float(*x22t)[kQ] = x11t + 64;                                    // x22t[k][c] = X22[c][k]
    float(*l21t)[kQ] = x22t + 64;                                    // l21t[k][c] = L21[c][k]
    float(*a1)[kQ] = l21t + 64;   // A[:, 0:64], then L[:, 0:64]
    float(*a2)[kQ] = a1 + 64;     // A[:, 64:128], then T, then L[:, 64:128]
    const int tid = threadIdx.x;
    const int64_t t0 = j0 + kP;
    const int64_t r0 = t0 + (int64_t)blockIdx.x * kPanelRows;
    for (int e = tid; e < 64 * 64; e += 256) {
        const int c = e >> 6, k = e & 63;
        x11t[k][c] = Pinv[e];
        x22t[k][c] = Pinv[64 * 64 + e];
        l21t[k][c] = Pinv[2 * 64 * 64 + e];
    }
    for (int e = tid; e < kPanelRows * kP; e += 256) {
        const int r = e >> 7, k = e & 127;
        const float v = r0 + r < n ? A[(r0 + r) * n + j0 + k] : 0.f;
        if (k < 64) a1[r][k] = v; else a2[r][k - 64] = v;
    }
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;
    float acc[4][4];
    // L1 = A1 X11^T
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = 0.f;
    panel_gemm64(a1, x11t, acc, ty, tx);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) a1[4 * ty + p][4 * tx + q] = acc[p][q];
    __syncthreads();
    // T = A2 - L1 L21^T
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = 0.f;
    panel_gemm64(a1, l21t, acc, ty, tx);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) a2[4 * ty + p][4 * tx + q] -= acc[p][q];
    __syncthreads();
    // L2 = T X22^T
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[p][q] = 0.f;
    panel_gemm64(a2, x22t, acc, ty, tx);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
        for (int q = 0; q < 4; q++) a2[4 * ty + p][4 * tx + q] = acc[p][q];
    __syncthreads();
    // stores: A rows (lanes along the row) and the TF32 hi / lo operand rows
    for (int e = tid; e < kPanelRows * kP; e += 256) {
        const int r = e >> 7, k = e & 127;
        const int64_t i = r0 + r;
        if (i >= n) continue;
        const float v = k < 64 ? a1[r][k] : a2[r][k - 64];
        A[i * n + j0 + k] = v;
        const float hi = tf32_rna(v);
        Whi[(i - t0) * kP + k] = hi;
        Wlo[(i - t0) * kP + k] = tf32_rna(v - hi);
    }
}

// ------------------------------- trailing update ----------------------------------
// tile index x -> (I, J), I >= J, x = I (I + 1) / 2 + J
__device__ __forceinline__ void tri_decode(int x, int &I, int &J) {
    int i = (int)((sqrtf(8.f * (float)x + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= x) i++;
    while (i * (i + 1) / 2 > x) i--;
    I = i;
    J = x - i * (i + 1) / 2;
}

// tile x of a launch -> (I, J).  mode 0: every tile I >= J; 1: the first block column (J = 0,
// the next panel's columns); 2: every tile 1 <= J <= I (the rest); 3: the first block column
// below its diagonal tile (I >= 1, J = 0)
__device__ __forceinline__ void tile_of(int x, int mode, int &I, int &J) {
    if (mode == 1 || mode == 3) {
        I = mode == 3 ? x + 1 : x;
        J = 0;
        return;
    }
    tri_decode(x, I, J);
    if (mode == 2) {
        I++;
        J++;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// named barrier of the sixteen epilogue warps (id 1; 0 is __syncthreads)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }
// a global load that is not made when `pred` is false (predicated PTX: no access at all), 0
// then; the L1-cached path, not the read-only one (the kernel writes A)
__device__ __forceinline__ float ld_if(const float *p, bool pred) {
    float x = 0.f;
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t@q ld.global.f32 %0, [%2];\n\t}"
        : "+f"(x)
        : "r"((int)pred), "l"(p));
    return x;
}

// Persistent trailing update: CTA c takes tiles c, c + gridDim.x, ...  Warp 0 streams the
// operands of its tiles through the two-stage TMA ring, warp 1 issues the MMAs of tile i
// into TMEM accumulator i % 2 (256 columns: two 128 x 128 FP32 accumulators), warps 2-17
// (four per TMEM lane quadrant, each a quarter of the columns) run the epilogue of tile i while the
// MMAs of tile i + 1 proceed: C(i), fetched into registers during tile i - 1, goes to shared
// memory, the fetch of C(i + 1) is issued, then wait for the accumulator, C -= X in shared
// memory, free the accumulator, write C back: each fetch has a whole tile's epilogue to
// arrive.  The fetch and the write-back go row by row (a warp per row, its lanes along the
// row: one row pointer per row, each instruction 128 consecutive bytes; A's rows start on
// any 4-byte boundary).  A CTA reads only its own tiles, each before it writes it.  Every
// mbarrier wait is
// bounded; a role that gives up records ERR_CHOL and the others give up on their next wait.
__global__ void __launch_bounds__(kTrailThreads, 1) k_cholp_trail(
    const __grid_constant__ CUtensorMap mHi, const __grid_constant__ CUtensorMap mLo, float *A,
    int64_t n, int64_t t0, int mode, int ntiles, int32_t *err) {
    extern __shared__ __align__(1024) unsigned char sm_trail[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(sm_trail) + 1023) & ~(uintptr_t)1023);
    float *Cs = reinterpret_cast<float *>(base + kStages * kStage);   // [128][129]
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kStages * kStage + kCsBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    __shared__ int s_fail;    // producer / MMA gave up (read only as an early exit)
    __shared__ int s_efail;   // an epilogue wait gave up: written by the epilogue warps before
                              // a named barrier and read after it, so all four exit together
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int nk = kP / 32;   // K steps of 32 TF32 columns (one 128-byte swizzle row)
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[kStages]);
    const uint32_t accf0 = smem_u32(&bars[2 * kStages]), acce0 = smem_u32(&bars[2 * kStages + 2]);
    if (threadIdx.x == 0) {
        s_fail = 0;
        s_efail = 0;
        for (int st = 0; st < kStages; st++) {
            mbar_init(full0 + 8 * st, 1);
            mbar_init(empty0 + 8 * st, 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, kEpiThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2 * 128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const int ntl = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (warp == 0 && lane == 0) {
        for (int i = 0; i < ntl && !s_fail; i++) {
            int I, J;
            tile_of((int)blockIdx.x + i * (int)gridDim.x, mode, I, J);
            for (int k = 0; k < nk; k++) {
                const int q = i * nk + k, st = q & 1;
                if (q >= 2 && !mbar_wait(empty0 + 8 * st, ((q >> 1) - 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                uint8_t *sp = base + st * kStage;
                const uint32_t bar = full0 + 8 * st;
                mbar_expect_tx(bar, kStage);
                tma_load_2d(smem_u32(sp), &mHi, 32 * k, 128 * I, bar);
                tma_load_2d(smem_u32(sp + kTile), &mLo, 32 * k, 128 * I, bar);
                tma_load_2d(smem_u32(sp + 2 * kTile), &mHi, 32 * k, 128 * J, bar);
                tma_load_2d(smem_u32(sp + 3 * kTile), &mLo, 32 * k, 128 * J, bar);
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_mma(128, 128, 2u);
        for (int i = 0; i < ntl && !s_fail; i++) {
            const int b = i & 1;
            if (i >= 2 && !mbar_wait(acce0 + 8 * b, ((i >> 1) - 1) & 1)) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t d = tmem + (uint32_t)(b * 128);
            for (int k = 0; k < nk; k++) {
                const int q = i * nk + k, st = q & 1;
                if (!mbar_wait(full0 + 8 * st, (q >> 1) & 1)) {
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sp = smem_u32(base + st * kStage);
                const uint32_t aH = sp, aL = sp + kTile, bH = sp + 2 * kTile, bL = sp + 3 * kTile;
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {   // 32 bytes (8 TF32) per MMA
                    const uint32_t off = ks * 32;
                    umma<false>(d, umma_desc_sw128(aH + off), umma_desc_sw128(bH + off), idesc,
                                (k > 0 || ks > 0) ? 1u : 0u);
                    umma<false>(d, umma_desc_sw128(aH + off), umma_desc_sw128(bL + off), idesc, 1u);
                    umma<false>(d, umma_desc_sw128(aL + off), umma_desc_sw128(bH + off), idesc, 1u);
                }
                umma_commit(empty0 + 8 * st);
            }
            umma_commit(accf0 + 8 * b);
        }
    } else if (warp >= 2) {
        const int ew = warp - 2;                     // epilogue warp 0 .. 15
        const int quad = warp & 3;                   // TMEM lane quadrant of this warp
        const int qcol = ew >> 2;                    // columns [32 qcol, 32 qcol + 32)
        const int row = quad * 32 + lane;            // tile row = TMEM lane
        // the next tile's C in registers: rows ew + 16 k, columns lane + 32 q (only its valid
        // elements are read: rows below n, columns below n and, on a diagonal tile, up to the
        // diagonal)
        float cn[8][4];
        auto fetch = [&](int i) {
            int I, J;
            tile_of((int)blockIdx.x + i * (int)gridDim.x, mode, I, J);
            const int64_t gr0 = t0 + 128 * (int64_t)I, gc0 = t0 + 128 * (int64_t)J;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int64_t gr = gr0 + ew + 16 * k;
                const int64_t cend = gr < n ? (I == J ? gr + 1 : n) - gc0 : 0;
                const float *src = A + gr * n + gc0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int c = lane + 32 * q;
                    cn[k][q] = ld_if(src + c, c < cend && gc0 + c < n);
                }
            }
        };
        if (ntl > 0) fetch(0);
        for (int i = 0; i < ntl; i++) {
            int I, J;
            tile_of((int)blockIdx.x + i * (int)gridDim.x, mode, I, J);
            const int64_t gr0 = t0 + 128 * (int64_t)I, gc0 = t0 + 128 * (int64_t)J;
            // C(i) into shared memory (Cs is free: the previous tile was written back)
#pragma unroll
            for (int k = 0; k < 8; k++)
#pragma unroll
                for (int q = 0; q < 4; q++) Cs[(ew + 16 * k) * kCsLd + lane + 32 * q] = cn[k][q];
            if (i + 1 < ntl) fetch(i + 1);
            const int b = i & 1;
            const bool got = mbar_wait(accf0 + 8 * b, (i >> 1) & 1);
            if (!got) s_efail = 1;
            epi_sync();
            if (s_efail) break;   // the same value for all epilogue threads (see s_efail)
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int cb = 0; cb < 32; cb += 16) {
                const int c0 = 32 * qcol + cb;
                float v[16];
                tmem_ld16(tmem + (uint32_t)(b * 128) + ((uint32_t)(quad * 32) << 16) + c0, v);
#pragma unroll
                for (int q = 0; q < 16; q++) Cs[row * kCsLd + c0 + q] -= v[q];
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(acce0 + 8 * b);   // the accumulator is free for tile i + 2
            epi_sync();
            for (int r = ew; r < 128; r += 16) {
                const int64_t gr = gr0 + r;
                if (gr >= n) break;
                const int64_t cend = (I == J ? gr + 1 : n) - gc0;
                float *dstg = A + gr * n + gc0;
                const float *srcs = Cs + r * kCsLd;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int c = lane + 32 * q;
                    if (c < cend && gc0 + c < n) dstg[c] = srcs[c];
                }
            }
            epi_sync();   // Cs is read out before the next tile's rows arrive
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && (s_fail || s_efail)) atomicAdd(&err[ERR_CHOL], 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(2 * 128));
}

// [rows][128] FP32 operand rows, boxes of 32 columns (one 128-byte swizzle row) x 128 rows
int make_w_map(CUtensorMap *map, float *base, int64_t rows) {
    auto enc = get_encode();
    if (!enc) return set_error(FEM3_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)kP, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kP * sizeof(float)};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FEM3_E_CUDA, "cuTensorMapEncodeTiled failed (factor)");
    return FEM3_OK;
}

// Side stream and events of the look-ahead, shared through a process-wide pool: a
// factorisation takes a context for the time it enqueues its launches (every wait on an
// event is enqueued before the event is recorded again), so concurrent callers never share
// one.
struct CholCtx {
    int device = -1;
    cudaStream_t side = nullptr;   // bulk trailing updates
    cudaStream_t col = nullptr;    // the next panel's columns below its diagonal tile
    std::vector<cudaEvent_t> ev;
};
std::mutex g_ctx_mu;
std::vector<CholCtx *> g_ctx_free;

int ctx_acquire(CholCtx **out, int npan) {
    int dev = 0;
    FEM3_CUDA(cudaGetDevice(&dev));
    CholCtx *c = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_ctx_mu);
        for (size_t i = 0; i < g_ctx_free.size(); i++)
            if (g_ctx_free[i]->device == dev) {
                c = g_ctx_free[i];
                g_ctx_free.erase(g_ctx_free.begin() + i);
                break;
            }
    }
    if (!c) {
        c = new CholCtx();
        c->device = dev;
        cudaError_t e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->col, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            if (c->side) cudaStreamDestroy(c->side);
            delete c;
            return cuda_error(e, "cudaStreamCreateWithFlags");
        }
    }
    while ((int)c->ev.size() < 4 * npan) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        if (r != cudaSuccess) {
            std::lock_guard<std::mutex> lk(g_ctx_mu);
            g_ctx_free.push_back(c);
            return cuda_error(r, "cudaEventCreateWithFlags");
        }
        c->ev.push_back(e);
    }
    *out = c;
    return FEM3_OK;
}

void ctx_release(CholCtx *c) {
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    g_ctx_free.push_back(c);
}

}  // namespace

// FP32 factorisation of A (n x n, lower triangle) in place, inverses of the 64 x 64
// diagonal blocks into m->dinv; the same output layout as the tile-task factorisation.
//
// Look-ahead over three streams.  Panel p: D(p) diagonal block, P(p) panel solve into the
// operand buffer p % 2, Ta(p) the trailing update of panel p + 1's diagonal tile, Tc(p) that
// of the rest of panel p + 1's columns, Tb(p) the rest of the trailing update.  The caller's
// stream runs D, P and Ta (the critical chain), the column stream Tc and the side stream Tb,
// so Tc(p) overlaps D(p + 1) and Tb(p) overlaps D(p + 1) and P(p + 1).  Orderings: D(p) after
// Tb(p - 2) (which updated panel p's columns and read the operand buffer P(p) rewrites) and
// Ta(p - 1); P(p) after Tc(p - 1) (panel p's columns below the diagonal tile; Tc(p - 2),
// earlier on its stream, read the operand buffer P(p) rewrites); Ta(p) and Tc(p) after P(p)
// and Tb(p - 1) (which updated the same columns); Tb(p) after P(p); the caller's stream waits
// for the last Tb and Tc.
int chol_tc(Mesh *m, float *A, int64_t n) {
    if (n <= 0) return FEM3_OK;
    cudaStream_t s = m->stream;
    const int64_t wrows = std::max<int64_t>(128, (n + 127) / 128 * 128);
    if (!m->chol_w || m->chol_w_rows < wrows) {
        FEM3_TRY(dev_alloc(m, (void **)&m->chol_w, sizeof(float) * (4 * wrows * kP + 3 * 64 * 64)));
        m->chol_w_rows = wrows;
        // operand rows past the trailing matrix are read by the edge tiles' MMAs (their
        // products are masked in the epilogue): keep them finite
        FEM3_CUDA(cudaMemsetAsync(m->chol_w, 0, sizeof(float) * 4 * wrows * kP, s));
    }
    float *W[2][2] = {{m->chol_w, m->chol_w + wrows * kP},
                      {m->chol_w + 2 * wrows * kP, m->chol_w + 3 * wrows * kP}};
    float *Linv = m->chol_w + 4 * wrows * kP;   // [X11 | X22 | L21] of the current panel
    CUtensorMap maps[2][2];
    for (int b = 0; b < 2; b++)
        for (int h = 0; h < 2; h++) FEM3_TRY(make_w_map(&maps[b][h], W[b][h], wrows));
    static bool attr = false;
    if (!attr) {
        FEM3_CUDA(cudaFuncSetAttribute(k_cholp_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * kDiagSmemFloats)));
        FEM3_CUDA(cudaFuncSetAttribute(k_cholp_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(float) * 5 * 64 * kQ)));
        FEM3_CUDA(cudaFuncSetAttribute(k_cholp_trail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTrailSmem));
        attr = true;
    }
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        FEM3_CUDA(cudaGetDevice(&dev));
        FEM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int npan = (int)((n + kP - 1) / kP);
    CholCtx *cx = nullptr;
    FEM3_TRY(ctx_acquire(&cx, npan));
    cudaStream_t s1 = cx->side, s2 = cx->col;
    cudaEvent_t *evP = cx->ev.data(), *evB = evP + npan, *evQ = evB + npan, *evR = evQ + npan;
    float *dinv = reinterpret_cast<float *>(m->dinv);
    int st = FEM3_OK;
    int last_b = -1, last_r = -1;
    auto launch_ok = [&](const char *what) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess && st == FEM3_OK) st = cuda_error(e, what);
        return st == FEM3_OK;
    };
    kc_begin(m, KC_FACTOR);
    for (int p = 0; p < npan && st == FEM3_OK; p++) {
        const int64_t j0 = (int64_t)p * kP;
        const int nbp = (int)std::min<int64_t>(kP, n - j0);
        if (p >= 2 && cudaStreamWaitEvent(s, evB[p - 2], 0) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaStreamWaitEvent");
            break;
        }
        k_cholp_diag<<<1, 512, sizeof(float) * kDiagSmemFloats, s>>>(A, n, j0, nbp, dinv, Linv,
                                                                      m->err);
        note_launch(m);
        if (!launch_ok("k_cholp_diag")) break;
        const int64_t t0 = j0 + nbp, mt = n - t0;
        if (mt <= 0) break;
        const int b = p & 1;
        if (p >= 1 && cudaStreamWaitEvent(s, evR[p - 1], 0) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaStreamWaitEvent");
            break;
        }
        k_cholp_panel<<<(unsigned)((mt + kPanelRows - 1) / kPanelRows), 256,
                        sizeof(float) * 5 * 64 * kQ, s>>>(A, n, j0, Linv, W[b][0], W[b][1]);
        note_launch(m);
        if (!launch_ok("k_cholp_panel")) break;
        const int64_t T = (mt + 127) / 128;
        if (cudaEventRecord(evP[p], s) != cudaSuccess ||
            cudaStreamWaitEvent(s1, evP[p], 0) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaEventRecord");
            break;
        }
        const int64_t nb_rest = T * (T + 1) / 2 - T;
        if (nb_rest > 0) {
            const int g = (int)std::min<int64_t>(nb_rest, std::max(1, sms - kReservedSms));
            k_cholp_trail<<<g, kTrailThreads, kTrailSmem, s1>>>(maps[b][0], maps[b][1], A, n, t0, 2,
                                                               (int)nb_rest, m->err);
            note_launch(m);
            if (!launch_ok("k_cholp_trail")) break;
        }
        if (cudaEventRecord(evB[p], s1) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaEventRecord");
            break;
        }
        last_b = p;
        if (p >= 1 && cudaStreamWaitEvent(s, evB[p - 1], 0) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaStreamWaitEvent");
            break;
        }
        // Tc(p) on the column stream, after P(p) and Tb(p - 1) (both behind this point of the
        // caller's stream); then Ta(p), the one tile D(p + 1) waits for
        if (cudaEventRecord(evQ[p], s) != cudaSuccess ||
            cudaStreamWaitEvent(s2, evQ[p], 0) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaEventRecord");
            break;
        }
        if (T > 1) {
            k_cholp_trail<<<(unsigned)std::min<int64_t>(T - 1, kReservedSms), kTrailThreads,
                            kTrailSmem, s2>>>(maps[b][0], maps[b][1], A, n, t0, 3, (int)(T - 1),
                                              m->err);
            note_launch(m);
            if (!launch_ok("k_cholp_trail")) break;
        }
        if (cudaEventRecord(evR[p], s2) != cudaSuccess) {
            st = cuda_error(cudaGetLastError(), "cudaEventRecord");
            break;
        }
        last_r = p;
        k_cholp_trail<<<1, kTrailThreads, kTrailSmem, s>>>(maps[b][0], maps[b][1], A, n, t0, 1, 1,
                                                             m->err);
        note_launch(m);
        if (!launch_ok("k_cholp_trail")) break;
    }
    // join: the caller's stream continues after the side streams' last updates
    if (last_b >= 0 && cudaStreamWaitEvent(s, evB[last_b], 0) != cudaSuccess && st == FEM3_OK)
        st = cuda_error(cudaGetLastError(), "cudaStreamWaitEvent");
    if (last_r >= 0 && cudaStreamWaitEvent(s, evR[last_r], 0) != cudaSuccess && st == FEM3_OK)
        st = cuda_error(cudaGetLastError(), "cudaStreamWaitEvent");
    kc_end(m, KC_FACTOR);
    ctx_release(cx);
    return st;
}

}  // namespace fem3
