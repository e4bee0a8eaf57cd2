// Tensor-core contraction X_b = L_b^T W R_b (TF32 x 3 or BF16 x 3 split products, FP32
// accumulate) on sm_103a: TMA loads with 128-byte swizzle, tcgen05.mma issued by one
// thread, the accumulator in tensor memory, tcgen05.ld epilogue adding s K (X + X^T) into
// the lower triangle of the FP32 matrix.  Section 2.1 element sum restricted, bin by bin,
// to the Section 2.3 template.
//
// Operands.  The tables of one axis (FP64 accuracy, hi + lo FP32 pairs) are split into
// pairs v = hi + lo of TF32 (cvt.rna) or BF16 (round to nearest) values, with the Gauss
// weights folded into R; they are stored as four row-major arrays [n_tmpl rows][Kp] where
// row dof_off[b] + c is local dof c of bin b and column k its k-th Gauss point (zero for
// k >= G_b).  The product
//   X = Lhi Rhi^T + Lhi Rlo^T + Llo Rhi^T
// drops lo*lo and the rounding of lo: about 3 * 2^-22 relative per product for TF32
// (11-bit significands), 3 * 2^-16 for BF16 (8-bit significands).
//
// Tiles.  One CTA computes the 128 x N block (N <= BN) of X for rows
// [128 mt, 128 mt + 128) and columns [BN nt, BN nt + N) of one bin, BN = 128 or 256 (the
// tile width is tuned per problem size class at run time, see contract_tc).  K steps of
// 128 bytes (one swizzle row: 32 TF32 or 64 BF16 Gauss points) are loaded by TMA into one
// stage; each K step is four MMAs of 32 bytes (K = 8 TF32 or 16 BF16) per product.
//
// Epilogue.  A bin of at most 128 dofs has all of X in one CTA: the accumulator goes
// through shared memory (the free stage, rows XOR-swizzled by the row index so that rows
// and columns read without bank conflicts) and each pair adds X[r][c] + X[c][r] once, the
// lanes of a warp along one row of A.  Larger bins add each X element into the lower
// triangle straight from the tcgen05.ld registers.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

// one pipeline stage: the bins' K loops are short (3 to 5 steps), and a 64 or 96 KB stage
// lets three or two CTAs share an SM, each one's loads and epilogue overlapping the others'
constexpr int kBM = 128, kStages = 1;
constexpr int kBoxRows = 128;                  // rows of one TMA box
constexpr uint32_t kBoxBytes = kBoxRows * 128; // 16 KB
constexpr int kRowBytes = 128;                 // one K step: one 128-byte swizzle row
constexpr uint32_t kTileA = kBM * kRowBytes;   // 16 KB
template <int BN> struct TcCfg {
    static constexpr uint32_t kTileB = BN * kRowBytes;                 // 16 or 32 KB
    static constexpr uint32_t kStageBytes = 2 * kTileA + 2 * kTileB;   // 64 or 96 KB
    static constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256;
    static constexpr int kMinBlocks = BN == 128 ? 3 : 2;
};
constexpr int kTileWidths[2] = {256, 128};   // candidates of the tuner, index = tile slot
constexpr int kWaitLimit = 1 << 22;

#include "tc_ptx.cuh"

// hi + lo split of the value x + x2 (|x2| <= ulp(x)) into the operand type
template <class OT> struct Split;
template <> struct Split<float> {
    __device__ static void run(float x, float x2, float &h, float &l) {
        h = tf32_rna(x);
        l = tf32_rna((x - h) + x2);
    }
};
template <> struct Split<__nv_bfloat16> {
    __device__ static void run(float x, float x2, __nv_bfloat16 &h, __nv_bfloat16 &l) {
        h = __float2bfloat16_rn(x);
        l = __float2bfloat16_rn((x - __bfloat162float(h)) + x2);   // x - h is exact
    }
};

// ------------------------------- split kernel ------------------------------------
// One warp per template row (bin b, local dof c), lanes over the row's Gauss points:
// coalesced reads of the table row (hi + lo pairs).  Writes the operator-apply operand W R
// as hi + lo FP32 pairs in the table layout (the apply reads L from the table itself)
// and, when Lhi is given, the
// tensor-core operands (the TF32 or BF16 pairs of the same values, zero past the bin's
// Gauss points).  No FP64 arithmetic: W R is formed in double-float FP32 operations.
template <class OT>
__global__ void __launch_bounds__(256) k_split_ops(
    const float2 *__restrict__ tabL, const float2 *__restrict__ tabR,
    const int32_t *__restrict__ row_bin, const int32_t *__restrict__ dof_off,
    const int32_t *__restrict__ gp_off, const double *__restrict__ w_slot,
    const int64_t *__restrict__ tab_off, const int32_t *__restrict__ tab_ld,
    int64_t row_lo, int64_t n_rows, int Kp, OT *Lhi, OT *Llo, OT *Rhi, OT *Rlo, float2 *apR,
    int4 *rng, RowLists rl) {
    const int64_t row = row_lo + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n_rows) return;
    const int b = row_bin[row];
    const int c = (int)(row - dof_off[b]);
    const int g0 = gp_off[b], G = gp_off[b + 1] - g0;
    const int64_t src = tab_off[b] + (int64_t)c * tab_ld[b];
    const int64_t dst = row * (int64_t)Kp;
    // the GEMM reads a bin's operands up to G rounded to one 128-byte row (kbk Gauss points)
    const int kbk = 128 / (int)sizeof(OT);
    const int kend = Lhi ? min(Kp, (G + kbk - 1) / kbk * kbk) : G;
    // Gauss-point range [first, end) of the row's nonzeros in L and in W R; the nonzeros
    // themselves compacted in Gauss-point order (lanes in step: one ballot per 32 points)
    int lf = G, le = 0, rf = G, re = 0, nl = 0, nr = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int k0 = 0; k0 < kend; k0 += 32) {
        const int k = k0 + lane;
        OT lh = OT(0.f), ll = OT(0.f), rh = OT(0.f), rl2 = OT(0.f);
        float2 lv = make_float2(0.f, 0.f), rv = make_float2(0.f, 0.f);
        bool nzl = false, nzr = false;
        if (k < G) {
            const float2 lp = tabL[src + k], rp = tabR[src + k];
            const float a = lp.x, a2 = lp.y, r1 = rp.x, r2 = rp.y;
            float wh, wl;
            f64_split(w_slot[g0 + k], wh, wl);
            float sh = 0.f, sl = 0.f;
            df_fma(r1, r2, wh, wl, sh, sl);
            const float wr = sh + sl, wr2 = sl - (wr - sh);
            if (apR) apR[src + k] = make_float2(wr, wr2);
            lv = lp;
            rv = make_float2(wr, wr2);
            nzl = a != 0.f || a2 != 0.f;
            nzr = wr != 0.f || wr2 != 0.f;
            if (nzl) {
                lf = min(lf, k);
                le = k + 1;
            }
            if (nzr) {
                rf = min(rf, k);
                re = k + 1;
            }
            if (Lhi) {
                Split<OT>::run(a, a2, lh, ll);
                Split<OT>::run(wr, wr2, rh, rl2);
            }
        }
        if (Lhi && k < kend) {
            Lhi[dst + k] = lh;
            Llo[dst + k] = ll;
            Rhi[dst + k] = rh;
            Rlo[dst + k] = rl2;
        }
        if (rl.g0) {
            const unsigned bl = __ballot_sync(0xffffffffu, nzl), br = __ballot_sync(0xffffffffu, nzr);
            if (nzl) {
                const int64_t o = src + nl + __popc(bl & below);
                rl.g0[o] = (uint16_t)k;
                rl.v0[o] = lv;
            }
            if (nzr) {
                const int64_t o = src + nr + __popc(br & below);
                rl.g1[o] = (uint16_t)k;
                rl.v1[o] = rv;
            }
            nl += __popc(bl);
            nr += __popc(br);
        }
    }
    lf = __reduce_min_sync(0xffffffffu, lf);
    le = __reduce_max_sync(0xffffffffu, le);
    rf = __reduce_min_sync(0xffffffffu, rf);
    re = __reduce_max_sync(0xffffffffu, re);
    if (lane == 0) {
        rng[row] = make_int4(le > 0 ? lf : 0, le, re > 0 ? rf : 0, re);
        if (rl.g0) {
            rl.n0[row] = nl;
            rl.n1[row] = nr;
        }
    }
}

// Gauss-point-major lists of the nonzeros of L and W R, one CTA per bin: warp w takes the
// chunks of 32 Gauss points w, w + 8, ... (lane = point), walks the rows in order (loads
// along the Gauss points, eight rows in flight) and appends (the row's index in the bin,
// value) to the point's list.  Entry k of point g = 32 c + l (chunk c of width w_c <= 32) sits
// at tab_off[b] + 32 c D_b + k w_c + l: the lanes of a chunk at the same entry are adjacent
// (coalesced stores here and loads in the apply), and the chunks fill the bin's D_b x ld_b
// block (w_c summed over the chunks is G_b <= ld_b).
constexpr int kGpRows = 8;
__global__ void __launch_bounds__(256) k_gp_lists(
    const float2 *__restrict__ tabL, const float2 *__restrict__ tabR,
    const double *__restrict__ w_slot, const int32_t *__restrict__ gp_off,
    const int32_t *__restrict__ dof_off,
    const int64_t *__restrict__ tab_off, const int32_t *__restrict__ tab_ld,
    uint16_t *__restrict__ rL, float2 *__restrict__ vL, int32_t *__restrict__ nL,
    uint16_t *__restrict__ rR, float2 *__restrict__ vR, int32_t *__restrict__ nR) {
    const int b = blockIdx.x;
    const int D = dof_off[b + 1] - dof_off[b];
    const int g0 = gp_off[b], G = gp_off[b + 1] - g0, ld = tab_ld[b];
    const int64_t t0 = tab_off[b];
    const float2 *L = tabL + t0, *R = tabR + t0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int gc = 32 * warp; gc < G; gc += 256) {
        const int g = gc + lane, wc = min(32, G - gc);
        if (g >= G) continue;
        const int64_t base = t0 + (int64_t)gc * D + lane;
        float wh, wl;   // the point's weight; W R formed as in k_split_ops (the same values)
        f64_split(w_slot[g0 + g], wh, wl);
        int nl = 0, nr = 0;
        for (int c0 = 0; c0 < D; c0 += kGpRows) {
            float2 a[kGpRows], w[kGpRows];
#pragma unroll
            for (int j = 0; j < kGpRows; j++) {
                const int c = min(c0 + j, D - 1);   // rows past D repeat the last (not used)
                a[j] = __ldg(L + (int64_t)c * ld + g);
                w[j] = __ldg(R + (int64_t)c * ld + g);
            }
#pragma unroll
            for (int j = 0; j < kGpRows; j++) {
                float sh = 0.f, sl = 0.f;
                df_fma(w[j].x, w[j].y, wh, wl, sh, sl);
                const float wr = sh + sl;
                w[j] = make_float2(wr, sl - (wr - sh));
            }
#pragma unroll
            for (int j = 0; j < kGpRows; j++) {
                if (c0 + j >= D) break;
                if (a[j].x != 0.f || a[j].y != 0.f) {
                    rL[base + (int64_t)nl * wc] = (uint16_t)(c0 + j);
                    vL[base + (int64_t)nl * wc] = a[j];
                    nl++;
                }
                if (w[j].x != 0.f || w[j].y != 0.f) {
                    rR[base + (int64_t)nr * wc] = (uint16_t)(c0 + j);
                    vR[base + (int64_t)nr * wc] = w[j];
                    nr++;
                }
            }
        }
        nL[g0 + g] = nl;
        nR[g0 + g] = nr;
    }
}

// ------------------------------- GEMM kernel --------------------------------------
struct TcWork {
    int bin, mt, nt, pad;
};

template <bool BF16, int BN>
__global__ void __launch_bounds__(128, TcCfg<BN>::kMinBlocks) k_contract_tc(
    const __grid_constant__ CUtensorMap mLhi, const __grid_constant__ CUtensorMap mLlo,
    const __grid_constant__ CUtensorMap mRhi, const __grid_constant__ CUtensorMap mRlo,
    const int4 *__restrict__ work, const int32_t *__restrict__ dof_off,
    const int32_t *__restrict__ dof_idx, const int32_t *__restrict__ gp_off, float sK, float *A,
    int64_t n_dof, int full, int32_t *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned tile area (swizzle atoms), barriers after it
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t kTileB = TcCfg<BN>::kTileB, kStageBytes = TcCfg<BN>::kStageBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kStages * kStageBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 1);
    __shared__ int s_fail;

    const int4 wk = work[blockIdx.x];
    const int bin = wk.x, mt = wk.y, nt = wk.z;
    const int row0 = dof_off[bin];
    const int D = dof_off[bin + 1] - row0;
    const int G = gp_off[bin + 1] - gp_off[bin];
    const int nvalid = min(BN, D - nt * BN);            // columns of this tile
    const int N = (nvalid + 15) & ~15;                  // MMA N: multiple of 16, <= BN
    constexpr int kBK = BF16 ? 64 : 32;                 // Gauss points per K step
    const int nk = (G + kBK - 1) / kBK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const uint32_t full0 = smem_u32(&bars[0]);          // full[s]  = bars[s]
    const uint32_t empty0 = smem_u32(&bars[kStages]);   // empty[s] = bars[kStages + s]
    const uint32_t done = smem_u32(&bars[2 * kStages]);
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; s++) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0 && nk > 0) {
        // producer: TMA loads into the stage ring
        for (int k = 0; k < nk; k++) {
            const int s = k % kStages;
            if (k >= kStages) {
                if (!mbar_wait(empty0 + 8 * s, ((k / kStages) - 1) & 1)) { s_fail = 1; break; }
            }
            uint8_t *st = base + s * kStageBytes;
            const uint32_t bar = full0 + 8 * s;
            const int nbox = (N + kBoxRows - 1) / kBoxRows;   // 128-row boxes of each B operand
            mbar_expect_tx(bar, 2 * kTileA + 2 * nbox * kBoxBytes);
            const int x = k * kBK;
            const int ya = row0 + mt * kBM, yb = row0 + nt * BN;
            tma_load_2d(smem_u32(st), &mLhi, x, ya, bar);
            tma_load_2d(smem_u32(st + kTileA), &mLlo, x, ya, bar);
            for (int h = 0; h < nbox; h++) {
                tma_load_2d(smem_u32(st + 2 * kTileA + h * kBoxBytes), &mRhi, x, yb + h * kBoxRows,
                            bar);
                tma_load_2d(smem_u32(st + 2 * kTileA + kTileB + h * kBoxBytes), &mRlo, x,
                            yb + h * kBoxRows, bar);
            }
        }
    } else if (warp == 1 && lane == 0 && nk > 0) {
        // MMA issuer
        const uint32_t idesc = idesc_mma(kBM, N, BF16 ? 1u : 2u);
        for (int k = 0; k < nk; k++) {
            const int s = k % kStages;
            if (!mbar_wait(full0 + 8 * s, (k / kStages) & 1)) { s_fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t st = smem_u32(base + s * kStageBytes);
            const uint32_t aH = st, aL = st + kTileA, bH = st + 2 * kTileA, bL = st + 2 * kTileA + kTileB;
#pragma unroll
            for (int ks = 0; ks < kRowBytes / 32; ks++) {   // 32 bytes per MMA K step
                const uint32_t off = ks * 32;
                const uint32_t acc = (k > 0 || ks > 0) ? 1u : 0u;
                umma<BF16>(tmem, umma_desc_sw128(aH + off), umma_desc_sw128(bH + off), idesc, acc);
                umma<BF16>(tmem, umma_desc_sw128(aH + off), umma_desc_sw128(bL + off), idesc, 1u);
                umma<BF16>(tmem, umma_desc_sw128(aL + off), umma_desc_sw128(bH + off), idesc, 1u);
            }
            umma_commit(empty0 + 8 * s);   // frees the stage when these MMAs finish
        }
        umma_commit(done);
    }
    __syncthreads();
    // epilogue: every warp waits for the accumulator; one outcome for the whole CTA
    const bool ok = __syncthreads_and((nk > 0) && mbar_wait(done, 0) && !s_fail);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) {
        if (threadIdx.x == 0 && nk > 0) atomicAdd(&err[ERR_TC], 1);
    } else if (full) {
        // general form: X itself (rows: the A operand's dofs, columns: the B operand's), no
        // symmetric fold, straight from the tcgen05.ld registers
        const int c1 = mt * kBM + warp * 32 + lane;
        const bool row_ok = c1 < D;
        const int64_t j1 = row_ok ? dof_idx[row0 + c1] : 0;
        for (int cb = 0; cb < N; cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
            if (!row_ok) continue;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                if (cb + q >= nvalid) break;
                atomicAdd(&A[j1 * n_dof + dof_idx[row0 + nt * BN + cb + q]], sK * v[q]);
            }
        }
    } else if (D <= kBM) {
        // the stage is free (every load was consumed by an MMA that has completed):
        // Xs[r][c] at r * 128 + (c ^ (r & 31)), 64 KB
        float *Xs = reinterpret_cast<float *>(base);
        const int r1 = warp * 32 + lane;
        for (int cb = 0; cb < N; cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
#pragma unroll
            for (int q = 0; q < 16; q++) Xs[r1 * kBM + ((cb + q) ^ lane)] = v[q];
        }
        __syncthreads();
        // A = sK (X + X^T) on the lower triangle, once per pair (2 X[r][r] on the diagonal)
        for (int r = warp; r < D; r += 4) {
            const int64_t jr = dof_idx[row0 + r];
            for (int c = lane; c <= r; c += 32) {
                const float x = Xs[r * kBM + (c ^ (r & 31))] + Xs[c * kBM + (r ^ (c & 31))];
                const int64_t jc = dof_idx[row0 + c];
                atomicAdd(&A[(jr > jc ? jr : jc) * n_dof + (jr > jc ? jc : jr)], sK * x);
            }
        }
    } else {
        const int c1 = mt * kBM + warp * 32 + lane;     // local row (dof) of this thread
        const bool row_ok = c1 < D;
        const int64_t j1 = row_ok ? dof_idx[row0 + c1] : 0;
        for (int cb = 0; cb < N; cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cb, v);
            if (!row_ok) continue;
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const int c2 = nt * BN + cb + q;
                if (cb + q >= nvalid) break;
                const int64_t j2 = dof_idx[row0 + c2];
                // A = sK (X + X^T): X[c1][c2] and X[c2][c1] both land on the lower-triangle
                // element (the factorisation reads only the lower triangle); the diagonal
                // gets 2 X[c][c]
                const float x = (j1 == j2 ? 2.f : 1.f) * sK * v[q];
                atomicAdd(&A[(j1 > j2 ? j1 : j2) * n_dof + (j1 > j2 ? j2 : j1)], x);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

// ------------------------------- host side ----------------------------------------
// [rows][Kp] operand of 4-byte (TF32) or 2-byte (BF16) elements; boxes of one 128-byte
// swizzle row by 128 rows
int make_map(CUtensorMap *map, void *base, int64_t rows, int Kp, bool bf16) {
    auto enc = get_encode();
    if (!enc) return set_error(FEM3_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * esz};
    cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)kBM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     2, base, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FEM3_E_CUDA, "cuTensorMapEncodeTiled failed");
    return FEM3_OK;
}

}  // namespace

// Build the per-axis operand buffers and work lists once per mesh.
static int tc_prepare(Mesh *m) {
    if (m->tc_ready) return FEM3_OK;
    cudaStream_t s = m->stream;
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        int maxG = 0;
        for (int b = 0; b < B.n_bins; b++) maxG = std::max(maxG, B.h_gp_off[b + 1] - B.h_gp_off[b]);
        B.tc_maxG = maxG;
        // room for either operand type: Kp rounded to 64 Gauss points, 4 bytes each
        const int64_t rows = std::max<int64_t>(1, B.n_tmpl);
        const int64_t kp_max = std::max(64, (maxG + 63) / 64 * 64);
        for (int q = 0; q < 4; q++)
            FEM3_TRY(dev_alloc(m, &B.tc_op[q], sizeof(float) * rows * kp_max));
        // work lists of both tile widths: (bin, m-tile, n-tile)
        for (int w = 0; w < 2; w++) {
            const int bn = kTileWidths[w];
            std::vector<int4> &work = B.h_tc_work[w];
            work.clear();
            for (int b = 0; b < B.n_bins; b++) {
                int D = B.h_dof_off[b + 1] - B.h_dof_off[b];
                int G = B.h_gp_off[b + 1] - B.h_gp_off[b];
                if (D == 0 || G == 0) continue;
                for (int mt = 0; mt * kBM < D; mt++)
                    for (int nt = 0; nt * bn < D; nt++) work.push_back(make_int4(b, mt, nt, 0));
            }
            B.tc_n_work[w] = (int)work.size();
            FEM3_TRY(dev_alloc_t(m, &B.tc_work[w], std::max(1, B.tc_n_work[w])));
            if (B.tc_n_work[w])
                FEM3_CUDA(cudaMemcpyAsync(B.tc_work[w], work.data(), sizeof(int4) * work.size(),
                                          cudaMemcpyHostToDevice, s));
        }
    }
    static bool attr = false;
    if (!attr) {
        FEM3_CUDA(cudaFuncSetAttribute(k_contract_tc<false, 256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcCfg<256>::kSmemBytes));
        FEM3_CUDA(cudaFuncSetAttribute(k_contract_tc<true, 256>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcCfg<256>::kSmemBytes));
        FEM3_CUDA(cudaFuncSetAttribute(k_contract_tc<false, 128>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcCfg<128>::kSmemBytes));
        FEM3_CUDA(cudaFuncSetAttribute(k_contract_tc<true, 128>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)TcCfg<128>::kSmemBytes));
        attr = true;
    }
    m->tc_ready = true;
    return FEM3_OK;
}

// Tile-width tuner: the first tensor-core contraction of a problem size class (operand
// type, template rows and largest bin, both bucketed) times the GEMMs of every axis with
// each tile width (second of two runs, CUDA events) and keeps the faster; later meshes of
// the class use it.  fem3_options.tc_tile forces a width.
static std::mutex g_tile_mu;
static std::map<uint64_t, int> g_tile_choice;   // class -> tile slot

static uint64_t tile_class(const Mesh *m, bool bf16) {
    int64_t rows = 0;
    int maxg = 0;
    for (int a = 0; a < 3; a++) {
        rows += m->bins[a].n_tmpl;
        maxg = std::max(maxg, m->bins[a].tc_maxG);
    }
    int lg = 0;
    while ((int64_t(1) << lg) < rows) lg++;
    return (uint64_t)bf16 | ((uint64_t)lg << 1) | ((uint64_t)((maxg + 31) / 32) << 8);
}

// the GEMMs of the three axes with tile slot w (A32 accumulates: the caller zeroes it)
static int tc_gemms(Mesh *m, bool bf16, int w, const CUtensorMap (*maps)[4], int only_axis = -1,
                    int full = 0) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    for (int axis = 0; axis < 3; axis++) {
        if (only_axis >= 0 && axis != only_axis) continue;
        AxisBins &B = m->bins[axis];
        // the work items of this part's bins: the list is in bin order
        int b0, b1;
        part_bins(m, axis, b0, b1);
        const std::vector<int4> &hw = B.h_tc_work[w];
        const auto lb = [&](int b) {
            return (int)(std::lower_bound(hw.begin(), hw.end(), b,
                                          [](const int4 &x, int v) { return x.x < v; }) -
                         hw.begin());
        };
        const int w0 = lb(b0), nw = lb(b1) - w0;
        if (nw <= 0) continue;
        const int4 *wk = B.tc_work[w] + w0;
        const CUtensorMap *mp = maps[axis];
        const float sk = full ? 1.0f : (float)m->sK[axis];
#define FEM3_TC_LAUNCH(BF, BN)                                                                  \
    k_contract_tc<BF, BN><<<nw, 128, TcCfg<BN>::kSmemBytes, s>>>(                              \
        mp[0], mp[1], mp[2], mp[3], wk, B.dof_off, B.dof_idx, B.gp_off, sk, m->A32, n, \
        full, m->err)
        if (kTileWidths[w] == 256) {
            if (bf16) FEM3_TC_LAUNCH(true, 256); else FEM3_TC_LAUNCH(false, 256);
        } else {
            if (bf16) FEM3_TC_LAUNCH(true, 128); else FEM3_TC_LAUNCH(false, 128);
        }
#undef FEM3_TC_LAUNCH
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int contract_tc(Mesh *m, bool bf16) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    FEM3_TRY(tc_prepare(m));
    double flops = 0;
    CUtensorMap maps[3][4];
    // the split of every axis first (the GEMMs below may run more than once when tuning)
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        for (int b = 0; b < B.n_bins; b++) {
            double D = B.h_dof_off[b + 1] - B.h_dof_off[b];
            double G = B.h_gp_off[b + 1] - B.h_gp_off[b];
            flops += 2.0 * D * D * G;
        }
        if (!B.tc_n_work[0]) continue;
        FEM3_TRY(ap_alloc(m, axis));
        const bool whole = m->nparts <= 1;   // a part's apply operands are not kept
        const int kbk = bf16 ? 64 : 32;   // Gauss points per 128-byte swizzle row
        const int Kp = std::max(kbk, (B.tc_maxG + kbk - 1) / kbk * kbk);
        // template rows of this part's bins (all rows unless assembled in parts)
        int b0, b1;
        part_bins(m, axis, b0, b1);
        const int64_t row_lo = B.h_dof_off[b0], row_hi = B.h_dof_off[b1];
        const unsigned grid = (unsigned)std::max<int64_t>(1, (row_hi - row_lo + 7) / 8);
        kc_begin(m, KC_SPLIT);
        if (bf16) {
            __nv_bfloat16 *op[4];
            for (int q = 0; q < 4; q++) op[q] = reinterpret_cast<__nv_bfloat16 *>(B.tc_op[q]);
            k_split_ops<__nv_bfloat16><<<grid, 256, 0, s>>>(
                m->tabL[axis], m->tabR[axis], B.row_bin, B.dof_off, B.gp_off, B.w_slot,
                B.tab_off, B.tab_ld, row_lo, row_hi, Kp, op[0], op[1], op[2], op[3], B.ap_R, B.ap_rng,
                whole ? row_lists(B) : RowLists{});
        } else {
            float *op[4];
            for (int q = 0; q < 4; q++) op[q] = reinterpret_cast<float *>(B.tc_op[q]);
            k_split_ops<float><<<grid, 256, 0, s>>>(
                m->tabL[axis], m->tabR[axis], B.row_bin, B.dof_off, B.gp_off, B.w_slot,
                B.tab_off, B.tab_ld, row_lo, row_hi, Kp, op[0], op[1], op[2], op[3], B.ap_R, B.ap_rng,
                whole ? row_lists(B) : RowLists{});
        }
        if (whole) launch_gp_lists(m, axis);
        kc_end(m, KC_SPLIT);
        note_launch(m);
        for (int q = 0; q < 4; q++)
            FEM3_TRY(make_map(&maps[axis][q], B.tc_op[q], B.n_tmpl, Kp, bf16));
    }
    // tile width: forced, cached for the size class, or tuned now
    int w = -1;
    m->tc_tuned = false;
    if (m->tc_tile_opt == 128 || m->tc_tile_opt == 256) {
        w = m->tc_tile_opt == 256 ? 0 : 1;
    } else if (m->nparts > 1) {
        w = 1;   // a part's GEMMs are not representative of the size class: no tuning
    } else {
        const uint64_t key = tile_class(m, bf16);
        {
            std::lock_guard<std::mutex> lk(g_tile_mu);
            auto it = g_tile_choice.find(key);
            if (it != g_tile_choice.end()) w = it->second;
        }
        if (w < 0) {
            cudaEvent_t e0, e1;
            FEM3_CUDA(cudaEventCreate(&e0));
            FEM3_CUDA(cudaEventCreate(&e1));
            float best = 0.f;
            for (int c = 0; c < 2; c++)
                for (int rep = 0; rep < 2; rep++) {
                    FEM3_CUDA(cudaMemsetAsync(m->A32, 0, sizeof(float) * n * n, s));
                    FEM3_CUDA(cudaEventRecord(e0, s));
                    FEM3_TRY(tc_gemms(m, bf16, c, maps));
                    FEM3_CUDA(cudaEventRecord(e1, s));
                    FEM3_CUDA(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    FEM3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (rep == 1 && (w < 0 || ms < best)) {
                        best = ms;
                        w = c;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lk(g_tile_mu);
            g_tile_choice[key] = w;
            m->tc_tuned = true;
        }
    }
    m->tc_tile_used = kTileWidths[w];
    FEM3_CUDA(cudaMemsetAsync(m->A32, 0, sizeof(float) * n * n, s));
    kc_begin(m, KC_CONTRACT);
    FEM3_TRY(tc_gemms(m, bf16, w, maps));
    kc_end(m, KC_CONTRACT);
    m->contract_flops = flops;
    m->ap_ready = m->nparts <= 1;   // a part's split covers only its own bins' rows
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

namespace {
// ws[slot] = wc[gp_idx[slot]]: the form's weights in one axis's slot order
__global__ void k_gather_slots(const double *__restrict__ wc, const int32_t *__restrict__ gp_idx,
                               int64_t n, double *ws) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ws[i] = wc[gp_idx[i]];
}
}  // namespace

// General form (c D^a u, D^^b v) of one axis on the tensor cores: K = T^T diag(wc) S (T the
// test side's table, S the trial side's) with the split products of the precision, into
// A32 (cleared first); every tile of every bin, no symmetric fold.  wc_gp holds 2 n_gp
// values: the weights per Gauss point, then room for them in slot order.
int contract_tc_form(Mesh *m, int axis, bool test_right, double *wc_gp, bool bf16) {
    cudaStream_t s = m->stream;
    const int64_t n = m->n_dof;
    FEM3_TRY(tc_prepare(m));
    AxisBins &B = m->bins[axis];
    FEM3_CUDA(cudaMemsetAsync(m->A32, 0, sizeof(float) * n * n, s));
    if (!B.tc_n_work[0]) return FEM3_OK;
    FEM3_TRY(ap_alloc(m, axis));
    double *ws = wc_gp + m->n_gp;
    k_gather_slots<<<(unsigned)((m->n_gp + 255) / 256), 256, 0, s>>>(wc_gp, B.gp_idx, m->n_gp, ws);
    note_launch(m);
    const int kbk = bf16 ? 64 : 32;
    const int Kp = std::max(kbk, (B.tc_maxG + kbk - 1) / kbk * kbk);
    const unsigned grid = (unsigned)((B.n_tmpl + 7) / 8);
    const float2 *T = test_right ? m->tabR[axis] : m->tabL[axis];
    const float2 *S = test_right ? m->tabL[axis] : m->tabR[axis];
    kc_begin(m, KC_SPLIT);
    if (bf16) {
        __nv_bfloat16 *op[4];
        for (int q = 0; q < 4; q++) op[q] = reinterpret_cast<__nv_bfloat16 *>(B.tc_op[q]);
        k_split_ops<__nv_bfloat16><<<grid, 256, 0, s>>>(T, S, B.row_bin, B.dof_off, B.gp_off, ws,
                                                         B.tab_off, B.tab_ld, 0, B.n_tmpl, Kp,
                                                         op[0], op[1], op[2], op[3], B.ap_R, B.ap_rng,
                                                         RowLists{});
    } else {
        float *op[4];
        for (int q = 0; q < 4; q++) op[q] = reinterpret_cast<float *>(B.tc_op[q]);
        k_split_ops<float><<<grid, 256, 0, s>>>(T, S, B.row_bin, B.dof_off, B.gp_off, ws,
                                                B.tab_off, B.tab_ld, 0, B.n_tmpl, Kp, op[0],
                                                op[1], op[2], op[3], B.ap_R, B.ap_rng, RowLists{});
    }
    kc_end(m, KC_SPLIT);
    note_launch(m);
    CUtensorMap maps[3][4];
    for (int q = 0; q < 4; q++) FEM3_TRY(make_map(&maps[axis][q], B.tc_op[q], B.n_tmpl, Kp, bf16));
    const int w = m->tc_tile_opt == 256 ? 0 : 1;   // 128 columns unless 256 is forced
    m->tc_tile_used = kTileWidths[w];
    kc_begin(m, KC_CONTRACT);
    FEM3_TRY(tc_gemms(m, bf16, w, maps, axis, 1));
    kc_end(m, KC_CONTRACT);
    m->ap_ready = false;   // ap_R now holds the form's operand
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int ap_alloc(Mesh *m, int axis) {
    AxisBins &B = m->bins[axis];
    if (B.ap_rng) return FEM3_OK;
    const int64_t e = std::max<int64_t>(1, B.tab_elems), nt = std::max<int64_t>(1, B.n_tmpl);
    const int64_t ng = std::max<int64_t>(1, m->n_gp);
    FEM3_TRY(dev_alloc(m, (void **)&B.ap_rng, sizeof(int4) * nt));
    if (!apply_lists_fit(m)) {   // the dense apply's W R operand instead of the lists
        FEM3_TRY(dev_alloc(m, (void **)&B.ap_R, sizeof(float2) * e));
        return FEM3_OK;
    }
    for (int t = 0; t < 2; t++) {
        FEM3_TRY(dev_alloc(m, (void **)&B.rl_g[t], sizeof(uint16_t) * e));
        FEM3_TRY(dev_alloc(m, (void **)&B.rl_v[t], sizeof(float2) * e));
        FEM3_TRY(dev_alloc(m, (void **)&B.rl_n[t], sizeof(int32_t) * nt));
        FEM3_TRY(dev_alloc(m, (void **)&B.gl_r[t], sizeof(uint16_t) * e));
        FEM3_TRY(dev_alloc(m, (void **)&B.gl_v[t], sizeof(float2) * e));
        FEM3_TRY(dev_alloc(m, (void **)&B.gl_n[t], sizeof(int32_t) * ng));
    }
    return FEM3_OK;
}

RowLists row_lists(AxisBins &B) {
    return RowLists{B.rl_g[0], B.rl_g[1], B.rl_v[0], B.rl_v[1], B.rl_n[0], B.rl_n[1]};
}

void launch_gp_lists(Mesh *m, int axis) {
    AxisBins &B = m->bins[axis];
    if (B.n_bins == 0 || !B.gl_r[0]) return;
    k_gp_lists<<<B.n_bins, 256, 0, m->stream>>>(m->tabL[axis], m->tabR[axis], B.w_slot,
                                                 B.gp_off, B.dof_off, B.tab_off, B.tab_ld,
                                                 B.gl_r[0], B.gl_v[0], B.gl_n[0], B.gl_r[1],
                                                 B.gl_v[1], B.gl_n[1]);
    note_launch(m);
}

// Operator-apply operands of the current tables, without the tensor-core operands.
int ap_prepare(Mesh *m) {
    if (m->ap_ready) return FEM3_OK;
    cudaStream_t s = m->stream;
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        if (B.n_tmpl == 0) continue;
        FEM3_TRY(ap_alloc(m, axis));
        kc_begin(m, KC_SPLIT);
        k_split_ops<float><<<(unsigned)((B.n_tmpl + 7) / 8), 256, 0, s>>>(
            m->tabL[axis], m->tabR[axis], B.row_bin, B.dof_off, B.gp_off, B.w_slot, B.tab_off,
            B.tab_ld, 0, B.n_tmpl, 0, nullptr, nullptr, nullptr, nullptr, B.ap_R, B.ap_rng,
            row_lists(B));
        launch_gp_lists(m, axis);
        kc_end(m, KC_SPLIT);
        note_launch(m);
    }
    m->ap_ready = true;
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

}  // namespace fem3
