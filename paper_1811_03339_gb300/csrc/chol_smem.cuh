// Device code of the dense Cholesky factorisation shared by the tile-task factorisation
// (solve.cu) and the blocked factorisation with tensor-core trailing updates (chol_tc.cu):
// release/acquire flag helpers, the FP32/FP64 reciprocal square root, and the 64 x 64
// diagonal-block factor-and-invert routine.  Included inside `namespace fem3 { namespace {`
// by each translation unit (every unit gets its own internal copy).

constexpr int NB = 64;   // block (tile) width of the factorisation

// ---------------------------------------------------------------------------------
// Cholesky
// ---------------------------------------------------------------------------------
constexpr int kSpinLimit = 1 << 22;   // x >= 64 ns sleep: > 0.25 s before giving up

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <class TF> __device__ __forceinline__ TF rsqrt_t(TF x);
// FP32: hardware estimate plus one Newton step y <- y + y (1 - x y^2) / 2, so that the
// factor is as accurate as one built from a correctly rounded square root (refinement
// then converges in as many sweeps).
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) {
    const float y = rsqrtf(x);
    const float r = fmaf(-x * y, y, 1.0f);
    return fmaf(0.5f * y, r, y);
}
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <class TF>
__device__ __forceinline__ void lds4(const TF *p, TF v[4]) {   // 16-byte aligned (float) / 32 (double)
    if constexpr (sizeof(TF) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2 *>(p);
        const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
        v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
    }
}
template <class TF>
__device__ __forceinline__ void lds2(const TF *p, TF v[2]) {
    if constexpr (sizeof(TF) == 4) {
        const float2 q = *reinterpret_cast<const float2 *>(p);
        v[0] = q.x; v[1] = q.y;
    } else {
        const double2 q = *reinterpret_cast<const double2 *>(p);
        v[0] = q.x; v[1] = q.y;
    }
}

constexpr int PB = 16;   // panel width inside the diagonal block

// named barriers of the diagonal factor (0 is __syncthreads)
constexpr int kBarPanelReady = 1;   // warp 0 -> update warps: block p factored and inverted
constexpr int kBarNextReady = 2;    // update warps -> warp 0: block p + 1 fully updated
constexpr int kBarUpdate = 3;       // among the 15 update warps
__device__ __forceinline__ void bar_sync_n(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int count) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// warp 0: 16 x 16 Cholesky of block p of a_s and its inverse in one pass.  Lanes 0..15 hold
// row r of the block (lower part), lanes 16..31 column r of the identity; step j broadcasts
// the pivot column (a_kj, k >= j, from lanes k) and every lane applies the same update,
// x_k -= (x_j / a_jj) a_kj (k > j), x_j /= sqrt(a_jj): on the rows this is the right-looking
// factorisation, on the identity's columns forward substitution with the new column of
// L_pp, so the inverse needs no pass of its own.  Entries above the diagonal of the row
// lanes are never read.  Writes L_pp into a_s, L_pp^{-1} into x_s and
// lt[k][c] = L_pp^{-1}[c][k].
template <class TF>
__device__ __forceinline__ void chol_inv16(TF (*a_s)[NB + 1], TF (*x_s)[NB + 1], TF (*lt)[PB + 4],
                                           int P, int nb, int64_t k0, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int r = lane & (PB - 1);
    const bool inv = lane >= PB;
    TF x[PB];
#pragma unroll
    for (int c = 0; c < PB; c++)
        x[c] = inv ? (c == r ? TF(1) : TF(0)) : (c <= r ? a_s[P + r][P + c] : TF(0));
    int bad = -1;
#pragma unroll
    for (int j = 0; j < PB; j++) {
        TF col[PB];
#pragma unroll
        for (int k = j; k < PB; k++) col[k] = __shfl_sync(0xffffffffu, x[j], k);
        const TF d = col[j];
        if (!(d > TF(0)) && bad < 0) bad = j;
        const TF rs = d > TF(0) ? rsqrt_t<TF>(d) : TF(1);
        const TF f = x[j] * rs * rs;
#pragma unroll
        for (int k = j + 1; k < PB; k++) x[k] -= f * col[k];
        x[j] *= rs;
    }
    if (bad >= 0 && lane == 0 && P + bad < nb)
        atomicCAS(&err[ERR_NOT_SPD], 0, (int32_t)(k0 + P + bad + 1));
    if (!inv) {
#pragma unroll
        for (int c = 0; c < PB; c++)
            if (c <= r) a_s[P + r][P + c] = x[c];
    } else {
#pragma unroll
        for (int i = 0; i < PB; i++) {
            x_s[P + i][P + r] = i >= r ? x[i] : TF(0);
            lt[r][i] = x[i];
        }
    }
}

// Diagonal block: factor A_kk = L_kk L_kk^T and form L_kk^{-1} (512 threads), blocked by
// 16 with look-ahead.  Warp 0 factors and inverts the 16 x 16 diagonal block p; 12 other
// warps then (a) solve the 16 rows of block p + 1 in panel p (L_{p+1,p} = A L_pp^{-T})
// and update diagonal block p + 1, which releases warp 0 for block p + 1 at once, and
// (b) meanwhile solve the rest of panel p, finish the inverse's block row p,
// (L^{-1})_pJ = -L_pp^{-1} T_pJ, apply the rest of the trailing update (2 x 2 blocks per
// thread) and form T_{p+1,J} = sum_K L_{p+1,K} (L^{-1})_KJ, which needs nothing of block
// p + 1 and so overlaps its factorisation.  The blocks of L^{-1} above the diagonal are
// zeroed first, while block 0 is factored.  a_s holds the block (rows and columns >= nb
// padded with the identity) and receives L (lower triangle); x_s receives L^{-1} in full
// (zero above the diagonal); the caller stores them.  A non-positive pivot records 1 + its
// global column (k0 + local).  Needs exactly 512 threads, all of the CTA; ends with a
// barrier.
template <class TF>
__device__ void potrf_inv_smem(TF (*a_s)[NB + 1], TF (*x_s)[NB + 1], int nb, int64_t k0,
                               int32_t *err) {
    // warps 4, 8 and 12 share warp 0's SM sub-partition and sit out: the 12 other warps
    // do the update work, so warp 0's serial factor competes with no issuing neighbour
    constexpr int NT = 416, NU = 384, NP = NB / PB;
    __shared__ __align__(16) TF lt[2][PB][PB + 4];     // lt[p & 1][k][c] = L_pp^{-1}[c][k]
    __shared__ __align__(16) TF pant[PB][NB + 4];      // pant[k][r] = L[r][P + k], r >= P + 16
    __shared__ __align__(16) TF tq[PB][NB - PB + 4];   // T_pJ, columns c < P
    const int tid = threadIdx.x;
    if (tid < 32) {
        for (int p = 0; p < NP; p++) {
            if (p > 0) bar_sync_n(kBarNextReady, NT);
            chol_inv16<TF>(a_s, x_s, lt[p & 1], p * PB, nb, k0, err);
            __syncwarp();
            bar_arrive_n(kBarPanelReady, NT);
        }
    } else if (((tid >> 5) & 3) != 0) {
        const int ut = ((tid >> 5) - 1 - (tid >> 7)) * 32 + (tid & 31);   // 0 .. NU - 1
        for (int e = ut; e < NB * NB; e += NU) {
            const int i = e >> 6, c = e & 63;
            if (c >= ((i >> 4) + 1) * PB) x_s[i][c] = TF(0);
        }
        for (int p = 0; p < NP; p++) {
            const int P = p * PB;
            bar_sync_n(kBarPanelReady, NT);
            const TF(*L16)[PB + 4] = lt[p & 1];
            // (a) block p + 1: its rows of panel p, then its diagonal update
            const int R0 = P + PB;
            if (p + 1 < NP) {
                TF xv = TF(0);
                const int xr = R0 + (ut >> 4), xc = ut & 15;
                if (ut < PB * PB) {
#pragma unroll
                    for (int k = 0; k < PB; k++) xv += a_s[xr][P + k] * L16[k][xc];
                }
                bar_sync_n(kBarUpdate, NU);
                if (ut < PB * PB) {
                    a_s[xr][P + xc] = xv;
                    pant[xc][xr] = xv;
                }
                bar_sync_n(kBarUpdate, NU);
                if (ut < PB * PB && xc + R0 <= xr) {
                    TF acc = TF(0);
#pragma unroll
                    for (int k = 0; k < PB; k++) acc += pant[k][xr] * pant[k][R0 + xc];
                    a_s[xr][R0 + xc] -= acc;
                }
                bar_arrive_n(kBarNextReady, NT);
            }
            // (b1) rows below block p + 1 (four columns per thread); the inverse's block
            // row p from T_pJ (formed in the previous panel)
            const int R1 = R0 + PB, m2 = NB - R1;
            const bool panel = m2 > 0 && ut < 4 * m2;
            const int pr = R1 + (ut >> 2), pc = (ut & 3) * 4;
            TF pv[4] = {TF(0), TF(0), TF(0), TF(0)};
            if (panel) {
#pragma unroll
                for (int k = 0; k < PB; k++) {
                    const TF av = a_s[pr][P + k];
                    TF lv[4];
                    lds4<TF>(&L16[k][pc], lv);
#pragma unroll
                    for (int q = 0; q < 4; q++) pv[q] += av * lv[q];
                }
            }
            TF iv[2] = {TF(0), TF(0)};
            if (p > 0) {
#pragma unroll
                for (int s2 = 0; s2 < 2; s2++) {
                    const int e = ut + NU * s2;
                    if (e < PB * P) {
                        const int i = e / P, c = e - i * P;
                        TF acc = TF(0);
#pragma unroll
                        for (int k = 0; k < PB; k++)
                            if (k <= i) acc += x_s[P + i][P + k] * tq[k][c];
                        iv[s2] = -acc;
                    }
                }
            }
            bar_sync_n(kBarUpdate, NU);
            // (b2) store the rows and the inverse's block row
            if (panel) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    a_s[pr][P + pc + q] = pv[q];
                    pant[pc + q][pr] = pv[q];
                }
            }
            if (p > 0) {
#pragma unroll
                for (int s2 = 0; s2 < 2; s2++) {
                    const int e = ut + NU * s2;
                    if (e < PB * P) {
                        const int i = e / P, c = e - i * P;
                        x_s[P + i][c] = iv[s2];
                    }
                }
            }
            if (p + 1 == NP) break;
            bar_sync_n(kBarUpdate, NU);
            // (b3) T_{p+1,J}[i][c] = sum_{k = c}^{R0 - 1} L[R0 + i][k] (L^{-1})[k][c], c < R0
            for (int e = ut; e < PB * R0; e += NU) {
                const int i = e / R0, c = e - i * R0;
                TF acc = TF(0);
                for (int kb = c & ~(PB - 1); kb < R0; kb += PB) {
#pragma unroll
                    for (int k = 0; k < PB; k++)
                        if (kb + k >= c) acc += a_s[R0 + i][kb + k] * x_s[kb + k][c];
                }
                tq[i][c] = acc;
            }
            // trailing update of blocks (i, k), i >= k >= p + 1, except block (p + 1, p + 1),
            // in 2 x 2 blocks (rows i0, i0 + 1 >= R1; columns j0, j0 + 1 >= R0)
            const int mr = (NB - R1) / 2, mc = (NB - R0) / 2;
            for (int e = ut; e < mr * mc; e += NU) {
                const int i0 = R1 + 2 * (e / mc), j0 = R0 + 2 * (e % mc);
                if (j0 > i0) continue;
                TF c00 = TF(0), c01 = TF(0), c10 = TF(0), c11 = TF(0);
#pragma unroll
                for (int k = 0; k < PB; k++) {
                    TF pi[2], pj[2];
                    lds2<TF>(&pant[k][i0], pi);
                    lds2<TF>(&pant[k][j0], pj);
                    c00 += pi[0] * pj[0];
                    c01 += pi[0] * pj[1];
                    c10 += pi[1] * pj[0];
                    c11 += pi[1] * pj[1];
                }
                a_s[i0][j0] -= c00;
                if (j0 + 1 <= i0) a_s[i0][j0 + 1] -= c01;
                a_s[i0 + 1][j0] -= c10;
                a_s[i0 + 1][j0 + 1] -= c11;
            }
        }
    }
    __syncthreads();
}
