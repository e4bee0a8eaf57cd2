// Path walk (Section 2.2) fused with the closed-form derivative tables (Section 2.1).
//
// One thread walks one (Gauss point, axis, side) ray x_g + r * dir * e_axis, r >= 0.
// In the current tet the ray's volume coordinates are b~ + r d~ with b~ = lambda_T(x_g)
// and d~ = dir * dlambda/dx_axis (eq. "cond"); the go-out parameter is
// r_max = min over d~_k < 0 of -b~_k / d~_k, and the zero pattern of b~ + r_max d~
// names the exit m-face (Fig. "fig:vc"): one zero -> the face neighbour, two -> an edge,
// three -> a vertex, in which case every tet holding the m-face is searched and the one
// the ray runs furthest into is taken (ties within eps_r: smallest id).
//
// On each segment [r_near, r_far] of tet T the left / right Riemann-Liouville
// derivative of order gamma of every local P1 basis function is added in closed form:
//   D_L:  + dphi/dx_axis |_T * (r_far^(1-gamma) - r_near^(1-gamma)) / Gamma(2-gamma)
//   D_R:  - (same)
// (integration by parts of eq. "def" on a segment where phi is linear; the end-point
// term phi(a) (x-a)^(-gamma)/Gamma(1-gamma) vanishes for interior basis functions).
// The sum telescopes over the path, so only one power r^(1-gamma) per segment end is
// evaluated.  Rows are accumulated in place in the thread's own column of its bin's
// table block [D_b][ld_b] (no two threads share an element).
#include <math.h>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

struct WalkGeom {
    const double *__restrict__ M;     // [T][16]
    const double *__restrict__ inv;   // [T][3][4]
    const float4 *__restrict__ rec;   // [T][3][8] FP32 records of the exit filter
    const int32_t *__restrict__ tets; // [T][4]
    const int32_t *__restrict__ nbr;  // [T][4]
    const int32_t *__restrict__ dof;  // [N]
    const int32_t *__restrict__ vt_off;
    const int32_t *__restrict__ vt_tet;
    const double *__restrict__ gp;    // [G][3]
    double eps_r;
    int max_steps;
};

// Monotone map of a double to a signed 64-bit key (same order as the doubles), so that
// comparisons and minima run on the integer pipes; the FP64 pipe is the scarce unit.
__device__ __forceinline__ long long ord_key(double v) {
    long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double key_double(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
// r < +inf (false for +inf and NaN), on the integer pipe
__device__ __forceinline__ bool below_inf(double r) {
    const long long b = __double_as_longlong(r);
    return b != 0x7FF0000000000000LL && (b & 0x7FFFFFFFFFFFFFFFLL) <= 0x7FF0000000000000LL;
}
// lambda <= eps for every non-NaN lambda, on the integer pipe: IEEE bit patterns of
// non-negative doubles are ordered like the values, negative ones are negative integers
__device__ __forceinline__ bool le_eps(double lam) {
    return __double_as_longlong(lam) <= __double_as_longlong(kEpsLambda);
}

// go-out parameter of the ray in tet t: min over exit candidates k (dir * dlambda_k/dx
// < 0, i.e. inv_k of the sign of -dir) of -b~_k / d~_k = -dir * b~_k * inv_k
__device__ __forceinline__ double tet_rmax(const WalkGeom &W, int32_t t, int axis, int dir,
                                           double x0, double x1, double x2, double b[4]) {
    const double2 *Mt = reinterpret_cast<const double2 *>(W.M + 16 * (int64_t)t);
    const double2 *ivp = reinterpret_cast<const double2 *>(W.inv + 12 * (int64_t)t + 4 * axis);
    const double2 iv0 = ivp[0], iv1 = ivp[1];
    const double ivk[4] = {iv0.x, iv0.y, iv1.x, iv1.y};
    long long kmin = ord_key(INFINITY);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        double2 a = Mt[2 * k], c = Mt[2 * k + 1];
        b[k] = fma(c.y, x2, fma(c.x, x1, fma(a.y, x0, a.x)));
        const long long ib = __double_as_longlong(ivk[k]);
        const bool cand = dir > 0 ? (ib < 0) : (ib > 0);
        if (cand) {
            double r = dir > 0 ? -(b[k] * ivk[k]) : b[k] * ivk[k];
            long long kr = ord_key(r);
            kmin = kr < kmin ? kr : kmin;
        }
    }
    return key_double(kmin);
}

// Per-line FP32 constants of the exit filter: the two coordinates across the axis,
// p1 = axis + 1 and p2 = axis + 2 (mod 3), as hi + lo pairs, and an upper bound of |x|_inf.
struct LineF {
    float xh1, xl1, xh2, xl2, xn;
};

__device__ __forceinline__ LineF line_f(double x0, double x1, double x2, int axis) {
    const double y1 = axis == 0 ? x1 : (axis == 1 ? x2 : x0);
    const double y2 = axis == 0 ? x2 : (axis == 1 ? x0 : x1);
    LineF X;
    X.xh1 = __double2float_rn(y1);
    X.xl1 = __double2float_rn(y1 - (double)X.xh1);
    X.xh2 = __double2float_rn(y2);
    X.xl2 = __double2float_rn(y2 - (double)X.xh2);
    X.xn = __double2float_ru(fmax(fabs(x0), fmax(fabs(x1), fabs(x2))));
    return X;
}

constexpr float kU32 = 5.9604644775390625e-08f;    // 2^-24, FP32 unit roundoff
constexpr float kTwoM44 = 5.684341886080802e-14f;  // 2^-44

// FP32 exit filter of one walk step (tet record R, ray direction dir along the axis).
// In the tet-local form of the record the ray meets lambda_k = 0 at the axis offset
// sigma_k = -beta_k / g_k from c_T, with beta_k = A_k + g_p1 dx_p1 + g_p2 dx_p2 and
// dx = x - c_T across the axis; the exit candidate (g_k of sign -dir) with the smallest
// dir * sigma_k is the exit, and lambda_k = beta_k + g_k sigma* at the exit gives the
// zero pattern.  Each quantity carries a bound on its distance from the value the FP64
// step computes: 16 u per magnitude for the FP32 rounding of the record, the split of x
// and the arithmetic (about 6 u needed), and F = 2^-44 (F0 + Gmax |x|_inf) for the FP64
// step's own rounding and the x split's second-order term (both below 2^-46 times that
// sum).  A decision is taken only where its bound separates it, so it is the FP64
// step's decision.  Returns false if some decision is within its bound (the caller then
// takes the FP64 step); else kstar = the exit candidate and zmask = the zero pattern
// without kstar's bit, which the caller tests in FP64.
__device__ __forceinline__ bool exit_filter(const float4 *__restrict__ R, const LineF &X, int dir,
                                            int &kstar, int &zmask) {
    const float4 A4 = __ldg(R), G4 = __ldg(R + 1), I4 = __ldg(R + 3), P4 = __ldg(R + 4),
                 Q4 = __ldg(R + 5), C4 = __ldg(R + 6);
    const float A[4] = {A4.x, A4.y, A4.z, A4.w}, G[4] = {G4.x, G4.y, G4.z, G4.w},
                I[4] = {I4.x, I4.y, I4.z, I4.w}, P[4] = {P4.x, P4.y, P4.z, P4.w},
                Q[4] = {Q4.x, Q4.y, Q4.z, Q4.w};
    const float d1 = (X.xh1 - C4.x) + X.xl1, d2 = (X.xh2 - C4.y) + X.xl2;
    const float F = kTwoM44 * fmaf(C4.w, X.xn, C4.z);
    float beta[4], eb[4], q[4], e[4];
    bool cand[4];
    float qs = INFINITY, es = 0.f;
    int ks = -1;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        beta[k] = fmaf(Q[k], d2, fmaf(P[k], d1, A[k]));
        const float S = fabsf(A[k]) + fabsf(P[k] * d1) + fabsf(Q[k] * d2);
        eb[k] = fmaf(16.f * kU32, S, F);
        const float sg = -beta[k] * I[k];
        q[k] = dir > 0 ? sg : -sg;
        e[k] = fmaf(fabsf(I[k]), eb[k], 4.f * kU32 * fabsf(sg));
        // the FP64 step's candidates: the sign bit of the reciprocal
        const int ib = __float_as_int(I[k]);
        cand[k] = dir > 0 ? ib < 0 : ib > 0;
        if (cand[k] && q[k] < qs) {
            qs = q[k];
            es = e[k];
            ks = k;
        }
    }
    if (ks < 0) return false;
    const float sig = dir > 0 ? qs : -qs;
    int zm = 0;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (k == ks) continue;
        if (cand[k] && !(q[k] - qs > e[k] + es)) ok = false;
        const float lam = fmaf(G[k], sig, beta[k]);
        const float El =
            eb[k] + F + fabsf(G[k]) * es + 4.f * kU32 * (fabsf(G[k] * sig) + fabsf(lam));
        if (lam <= 1e-12f - El)
            zm |= 1 << k;
        else if (!(lam > 1e-12f + El))
            ok = false;
    }
    kstar = ks;
    zmask = zm;
    return ok;
}

// One walk step in tet t: the go-out parameter r_max (the FP64 expression of tet_rmax)
// and the zero pattern of the volume coordinates there (FP64 test lambda <= eps_lambda),
// decided by the FP32 filter where its bounds allow and by the FP64 step otherwise, with
// the same outcome either way.  r_max = +inf if the ray cannot leave t.
__device__ __forceinline__ double exit_step(const WalkGeom &W, const LineF &X, int32_t t,
                                            int axis, int dir, double x0, double x1, double x2,
                                            int &zmask) {
    int ks, zm;
    if (exit_filter(W.rec + 8 * (3 * (int64_t)t + axis), X, dir, ks, zm)) {
        const double2 *Mk = reinterpret_cast<const double2 *>(W.M + 16 * (int64_t)t) + 2 * ks;
        const double2 a = Mk[0], c = Mk[1];
        const double bk = fma(c.y, x2, fma(c.x, x1, fma(a.y, x0, a.x)));
        const double iv = W.inv[12 * (int64_t)t + 4 * axis + ks];
        const double rmax = dir > 0 ? -(bk * iv) : bk * iv;
        // lambda_k* at r_max is b - fl(b fl(1/g)) g with one fused rounding: at most 2^-52 |b|,
        // below eps_lambda for |b| <= 4000 (an integer test); a larger |b| is tested in FP64
        bool zk = (__double_as_longlong(bk) & 0x7fffffffffffffffLL) <= 0x40AF400000000000LL;
        if (!zk) {
            const double gk = axis == 0 ? a.y : (axis == 1 ? c.x : c.y);
            zk = le_eps(fma(dir > 0 ? rmax : -rmax, gk, bk));
        }
        zmask = zm | (zk ? 1 << ks : 0);
        return rmax;   // finite: b and 1/g are
    }
    double b[4];
    const double rmax = tet_rmax(W, t, axis, dir, x0, x1, x2, b);
    const double *Mt = W.M + 16 * (int64_t)t;
    const double rs = dir > 0 ? rmax : -rmax;
    int z = 0;
#pragma unroll
    for (int k = 0; k < 4; k++)
        if (le_eps(fma(rs, Mt[4 * k + 1 + axis], b[k]))) z |= 1 << k;
    zmask = z;
    return rmax;
}

// next tet after leaving t at parameter rmax through the m-face of the zero pattern
// zmask; -1 at the boundary, -2 on a bad pattern
__device__ int32_t next_tet(const WalkGeom &W, int32_t t, int axis, int dir, double x0,
                            double x1, double x2, int zmask, double rmax) {
    int nz = __popc(zmask);
    if (nz == 1) return W.nbr[4 * (int64_t)t + (__ffs(zmask) - 1)];
    if (nz < 2 || nz > 3) return -2;
    // edge or vertex exit: search the star of the m-face
    int32_t fv[4];
    int nf = 0;
    for (int k = 0; k < 4; k++)
        if (!(zmask & (1 << k))) fv[nf++] = W.tets[4 * (int64_t)t + k];
    int32_t v0 = fv[0];
    double best = -INFINITY;
    int32_t next = -1;
    for (int pass = 0; pass < 2; pass++) {
        for (int32_t c = W.vt_off[v0]; c < W.vt_off[v0 + 1]; c++) {
            int32_t u = W.vt_tet[c];
            if (u == t) continue;
            bool has_all = true;
            for (int f = 1; f < nf; f++) {
                bool found = false;
                for (int q = 0; q < 4; q++) found |= W.tets[4 * (int64_t)u + q] == fv[f];
                has_all &= found;
            }
            if (!has_all) continue;
            double bu[4];
            double ru = tet_rmax(W, u, axis, dir, x0, x1, x2, bu);
            if (!(ru > rmax + W.eps_r)) continue;
            if (pass == 0) {
                best = fmax(best, ru);
            } else if (ru >= best - W.eps_r && (next < 0 || u < next)) {
                next = u;
            }
        }
    }
    return next;
}

// position of key j in the ascending list d[0 .. n), or -1: binary lifting for the number
// of entries <= j, with a trip count set by n alone (lanes searching one list stay
// converged) and every load inside the list
__device__ __forceinline__ int bsearch_key(const unsigned long long *__restrict__ d, int n,
                                           unsigned long long j) {
    if (n <= 0) return -1;
    int base = 0;
    for (int step = 1 << (31 - __clz(n)); step > 0; step >>= 1) {
        const int c = base + step;
        const unsigned long long v = __ldg(d + (c < n ? c : n) - 1);
        if (c <= n && v <= j) base = c;
    }
    return (base > 0 && __ldg(d + base - 1) == j) ? base - 1 : -1;
}

struct TableArgs {
    const int32_t *__restrict__ gp_idx;   // [n_gp] slot -> Gauss point
    const int32_t *__restrict__ slot_bin; // [n_gp]
    const int32_t *__restrict__ gp_off;   // [n_bins+1]
    const int32_t *__restrict__ dof_off;  // [n_bins+1]
    const unsigned long long *__restrict__ dof_key;   // template rows' keys (sorted per bin)
    const uint32_t *__restrict__ dof_q;               // [n_dof] position part of a dof's key
    const int64_t *__restrict__ tab_off;
    const int32_t *__restrict__ tab_ld;
    float2 *tab;                          // L (side 0) or R (side 1) of this axis, hi + lo pairs
    double p_exp;                         // 1 - gamma
    float coef_h, coef_l;                 // +1/Gamma(2-gamma) (left) or -1/Gamma(2-gamma), hi + lo
    const float2 *__restrict__ pow_cell;  // [256][8] local Taylor coefficients of m^p (hi + lo)
    const float2 *__restrict__ pow_exp;   // [128] 2^(e p) for e = -64 .. 63 (hi + lo)
};

// r^p for r > 0 by table-driven range reduction (after Tang's table-driven elementary
// functions): r = 2^e m with m in [1, 2); the top 8 fraction bits pick a cell of width
// 1/256 with centre m_c; m^p = sum_k C(p,k) m_c^(p-k) (m - m_c)^k, k <= 4, whose
// truncation error is below 1e-15 relative for p in [0, 1); 2^(e p) from a table.
// Evaluated in double-float FP32 arithmetic (hi + lo pairs, about 1e-14 relative): the
// range reduction is integer work and m - m_c is exact from the fraction bits, so the only
// FP64 operation is the rare fallback for exponents outside [-64, 63].
__device__ __forceinline__ void pow_df(double r, double p, const float2 *__restrict__ cell,
                                       const float2 *__restrict__ pexp, float &ph, float &pl) {
    const long long bits = __double_as_longlong(r);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    if (e < -64 || e > 63) {
        f64_split(pow(r, p), ph, pl);
        return;
    }
    const int j = (int)((bits >> 44) & 0xff);
    // m - m_c in units of 2^-52: the low 44 fraction bits minus the cell centre's 2^43
    const long long D = (bits & 0xFFFFFFFFFFFLL) - (1LL << 43);
    const float dh = small_int_f32((int)(D >> 21)) * 4.656612873077393e-10f;         // 2^-31
    const float dl = small_int_f32((int)(D & 0x1FFFFF)) * 2.220446049250313e-16f;    // 2^-52
    const float2 *c = cell + 8 * j;
    float2 ck = __ldg(c + 4);
    float qh = ck.x, ql = ck.y;
#pragma unroll
    for (int k = 3; k >= 0; k--) {
        df_mul(qh, ql, dh, dl, qh, ql);
        ck = __ldg(c + k);
        df_add2(qh, ql, ck.x, ck.y, qh, ql);
    }
    const float2 s = __ldg(pexp + e + 64);
    df_mul(qh, ql, s.x, s.y, ph, pl);
}

// entry k (0..7) of cell j of the power for exponent p: the Taylor term C(p,k) m_c^(p-k)
// for k <= 4 (zero for k >= 5), and from k = 5, for j < 128, 2^((j - 64) p); FP64 values
// stored as hi + lo pairs.  One thread per entry: the FP64 power is the slow part.
__device__ __forceinline__ void fill_pow_entry(double p, int j, int k, float2 *cell,
                                               float2 *pexp) {
    float h = 0.f, l = 0.f;
    if (k <= 4) {
        const double mc = 1.0 + (2.0 * j + 1.0) / 512.0;
        double binom = 1.0;
        for (int i = 0; i < k; i++) binom = binom * (p - i) / (i + 1);
        f64_split(binom * pow(mc, p - k), h, l);
    }
    cell[8 * j + k] = make_float2(h, l);
    if (k == 5 && j < 128) {
        f64_split(exp2((double)(j - 64) * p), h, l);
        pexp[j] = make_float2(h, l);
    }
}

// tables of the power for p = 1 - gamma_axis: cell[a][j][0..7], pexp[a][e + 64];
// grid (8 entries, 3 axes) x 256 cells
__global__ void k_pow_tables(double p0, double p1, double p2, float2 *cell, float2 *pexp) {
    const int k = blockIdx.x, a = blockIdx.y, j = threadIdx.x;
    const double p = a == 0 ? p0 : (a == 1 ? p1 : p2);
    fill_pow_entry(p, j, k, cell + (size_t)a * 256 * 8, pexp + a * 128);
}

// (table entry) += (h + l)
__device__ __forceinline__ void flush_entry(float2 *tab, int32_t col, int32_t ld, float h,
                                            float l) {
    float2 *te = tab + (int64_t)col * ld;
    float2 v = *te;
    df_add(h, l, v.x, v.y);
    *te = v;
}

// One line (Gauss point in slot `slot` of an axis): both directions in one loop.  When
// the left walk reaches the boundary the same iteration switches to the right walk, so a
// lane's trip count is one whole chord (nearly equal for neighbouring Gauss points) and
// the lanes of a warp stay converged.  The table entries of the current tet's vertices
// are accumulated in registers (consecutive tets of a path share three vertices) and
// added to the table when a vertex drops out of the current tet or the walk ends, so a
// step costs about one table read-modify-write.  Returns the number of segments; counts
// template misses and failed walks.
// Lines from `slot` on: after each line, next() gives the slot of another line or -1.  A
// lane that finishes its line takes the next one in the same loop, so the lanes of a warp
// stay busy until the lines run out instead of waiting for the warp's longest chord.
template <class Next>
__device__ __forceinline__ int walk_lines(const WalkGeom &W, const TableArgs &A0,
                                          const TableArgs &A1, int axis, int64_t slot,
                                          Next next, int &miss, int &bad) {
    int nseg = 0;
    int32_t g, nd, ld;
    const unsigned long long *dofs;
    int64_t toff;
    double x0, x1, x2;
    LineF X;
    int side, steps;   // side 0: left walk (dir -1, table L), 1: right walk (dir +1, table R)
    int32_t t;
    double r_prev;
    float pp_h, pp_l;   // r_prev^p
    auto begin_line = [&](int64_t sl) {
        g = A0.gp_idx[sl];
        const int32_t bin = A0.slot_bin[sl];
        const int32_t row = (int32_t)(sl - A0.gp_off[bin]);
        dofs = A0.dof_key + A0.dof_off[bin];
        nd = A0.dof_off[bin + 1] - A0.dof_off[bin];
        ld = A0.tab_ld[bin];
        toff = A0.tab_off[bin] + row;
        x0 = W.gp[3 * (int64_t)g];
        x1 = W.gp[3 * (int64_t)g + 1];
        x2 = W.gp[3 * (int64_t)g + 2];
        X = line_f(x0, x1, x2, axis);
        // this line's rows of L and R (no other thread writes them): zero before accumulating
        for (int c = 0; c < nd; c++) {
            A0.tab[toff + (int64_t)c * ld] = make_float2(0.f, 0.f);
            A1.tab[toff + (int64_t)c * ld] = make_float2(0.f, 0.f);
        }
        side = 0;
        steps = 0;
        t = g >> 2;
        r_prev = 0.0;
        pp_h = 0.f;
        pp_l = 0.f;
    };
    begin_line(slot);
    // live vertices: dof (-2: none), table column (-1: none), accumulated entry (hi + lo)
    int32_t sj[4] = {-2, -2, -2, -2}, sc[4] = {-1, -1, -1, -1};
    float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
    for (;;) {   // at most max_steps steps per side
        const int dir = side ? 1 : -1;
        float2 *const tab = (side ? A1.tab : A0.tab) + toff;
        const int4 tv = __ldg(reinterpret_cast<const int4 *>(W.tets) + t);
        int zmask;
        const double rmax = exit_step(W, X, t, axis, dir, x0, x1, x2, zmask);
        int32_t nx = -2;
        if (below_inf(rmax)) {
            nx = next_tet(W, t, axis, dir, x0, x1, x2, zmask, rmax);
            if (rmax - r_prev > W.eps_r) {
                // table part in double-float FP32: c = coef (rmax^p - r_prev^p)
                float ph, pl, ch, cl;
                // each side has its own order (unequal orders of the general form)
                pow_df(rmax, side ? A1.p_exp : A0.p_exp, side ? A1.pow_cell : A0.pow_cell,
                       side ? A1.pow_exp : A0.pow_exp, ph, pl);
                df_add2(ph, pl, -pp_h, -pp_l, ch, cl);
                df_mul(ch, cl, side ? A1.coef_h : A0.coef_h, side ? A1.coef_l : A0.coef_l, ch,
                       cl);
                // dlambda_v/dx_axis as hi + lo pairs from the tet's record
                const float4 *R = W.rec + 8 * (3 * (int64_t)t + axis);
                const float4 gh4 = __ldg(R + 1), gl4 = __ldg(R + 2);
                const float ghv[4] = {gh4.x, gh4.y, gh4.z, gh4.w},
                            glv[4] = {gl4.x, gl4.y, gl4.z, gl4.w};
                const int32_t j[4] = {W.dof[tv.x], W.dof[tv.y], W.dof[tv.z], W.dof[tv.w]};
                // slots kept (their dof is a vertex of t) and vertices already in a slot
                unsigned keep = 0, need = 0;
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    bool hit = false;
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (sj[q] == j[v]) {
                            hit = true;
                            keep |= 1u << q;
                        }
                    if (!hit && j[v] >= 0) need |= 1u << v;
                }
                // slots whose vertex left: the entries go to the table (one write per pass
                // for all lanes), then the slots are freed
                unsigned flw = 0;
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (!(keep & (1u << q)) && sc[q] >= 0) flw |= 1u << q;
                while (flw) {
                    const int q = __ffs(flw) - 1;
                    flw &= flw - 1;
                    const int32_t c = q == 0 ? sc[0] : (q == 1 ? sc[1] : (q == 2 ? sc[2] : sc[3]));
                    const float h = q == 0 ? sh[0] : (q == 1 ? sh[1] : (q == 2 ? sh[2] : sh[3]));
                    const float l = q == 0 ? sl[0] : (q == 1 ? sl[1] : (q == 2 ? sl[2] : sl[3]));
                    flush_entry(tab, c, ld, h, l);
                }
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (!(keep & (1u << q))) {
                        sj[q] = -2;
                        sc[q] = -1;
                        sh[q] = 0.f;
                        sl[q] = 0.f;
                    }
                // new vertices take free slots; one template search per pass for all lanes
                unsigned freem = ~keep & 0xFu;
                while (need) {
                    const int v = __ffs(need) - 1;
                    need &= need - 1;
                    const int q = __ffs(freem) - 1;
                    freem &= freem - 1;
                    const int32_t jv = v == 0 ? j[0] : (v == 1 ? j[1] : (v == 2 ? j[2] : j[3]));
                    const unsigned long long key =
                        ((unsigned long long)__ldg(A0.dof_q + jv) << 32) | (unsigned long long)jv;
                    const int32_t c = bsearch_key(dofs, nd, key);
#pragma unroll
                    for (int u = 0; u < 4; u++)
                        if (u == q) {
                            sj[u] = jv;
                            sc[u] = c;
                        }
                }
                // add c * dlambda_v/dx_axis to the slot of each vertex v
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (sj[q] < 0) continue;
                    float gh = ghv[0], gl = glv[0];
#pragma unroll
                    for (int v = 1; v < 4; v++)
                        if (sj[q] == j[v]) {
                            gh = ghv[v];
                            gl = glv[v];
                        }
                    if (sc[q] >= 0)
                        df_fma(ch, cl, gh, gl, sh[q], sl[q]);
                    else
                        miss++;
                }
                pp_h = ph;
                pp_l = pl;
                r_prev = rmax;
                nseg++;
            }
        }
        steps++;
        if (nx >= 0 && steps < W.max_steps) {
            t = nx;
            continue;
        }
        bad += (nx != -1);   // no exit found, bad pattern or step cap
        // end of this direction: the live entries go to the table
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (sc[q] >= 0) flush_entry(tab, sc[q], ld, sh[q], sl[q]);
            sj[q] = -2;
            sc[q] = -1;
            sh[q] = 0.f;
            sl[q] = 0.f;
        }
        if (side == 1) {
            const int64_t ns = next();
            if (ns < 0) break;
            begin_line(ns);
            continue;
        }
        // switch to the right walk of the same line (same order 1 - gamma on both sides)
        side = 1;
        t = g >> 2;
        r_prev = 0.0;
        pp_h = 0.f;
        pp_l = 0.f;
        steps = 0;
    }
    return nseg;
}

__device__ __forceinline__ int walk_line(const WalkGeom &W, const TableArgs &A0,
                                         const TableArgs &A1, int axis, int64_t slot,
                                         int &miss, int &bad) {
    return walk_lines(W, A0, A1, axis, slot, []() -> int64_t { return -1; }, miss, bad);
}

__device__ __forceinline__ void count_segments(int nseg, unsigned long long *seg_count) {
    unsigned long long ns = (unsigned long long)nseg;
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_down_sync(0xffffffffu, ns, o);
    if ((threadIdx.x & 31) == 0 && ns) atomicAdd(seg_count, ns);
}

// the three axes' table arguments (kernel parameters)
struct AxisTables {
    TableArgs A0[3], A1[3];
    int64_t lo[3], hi[3];   // the slots of each axis to walk, [lo, hi) (a bin range's slots)
};

// grid: x over blocks of `per_block` consecutive slots of an axis (bin order), y = axis; the
// three axes in one launch keep every SM filled.  A block's lanes start on its first 128
// lines and take the rest from a shared counter as they finish (per_block = 128 gives one
// line per lane).
__global__ void __launch_bounds__(128, 6) k_walk_tables(WalkGeom W, AxisTables T, int64_t n_gp,
                                                        int per_block, int axis0, int32_t *err,
                                                        unsigned long long *seg_count) {
    __shared__ int s_next;
    const int axis = axis0 + blockIdx.y;
    const int64_t base = T.lo[axis] + blockIdx.x * (int64_t)per_block;
    const int64_t end = min(base + per_block, T.hi[axis]);
    if (threadIdx.x == 0) s_next = blockDim.x;
    __syncthreads();
    const int64_t slot = base + threadIdx.x;
    int nseg = 0, miss = 0, bad = 0;
    if (slot < end) {
        auto next = [&]() -> int64_t {
            const int64_t sl = base + atomicAdd(&s_next, 1);
            return sl < end ? sl : -1;
        };
        nseg = walk_lines(W, T.A0[axis], T.A1[axis], axis, slot, next, miss, bad);
    }
    if (bad) atomicAdd(&err[ERR_WALK], bad);
    if (miss) atomicAdd(&err[ERR_TEMPLATE], miss);
    count_segments(nseg, seg_count);   // every lane takes part
}

// ---------------------------------------------------------------------------------
// Batched walk: one launch walks every line of every axis of every mesh in a batch.
// Descriptor d covers the n_gp slots of one (mesh, axis); item i belongs to the last
// descriptor with slot0 <= i.
// ---------------------------------------------------------------------------------
struct WalkDesc {
    WalkGeom W;
    TableArgs A0, A1;
    int axis;
    int64_t slot0, n_gp;
    int32_t *err;
    unsigned long long *seg;
};

__global__ void __launch_bounds__(128, 6) k_walk_batch(const WalkDesc *__restrict__ descs, int n_desc,
                                                    int64_t n_items) {
    const int64_t item = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int nseg = 0, miss = 0, bad = 0, d = 0;
    if (item < n_items) {
        int lo = 0, hi = n_desc - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].slot0 <= item) lo = mid; else hi = mid - 1;
        }
        d = lo;
        const WalkDesc &D = descs[d];
        nseg = walk_line(D.W, D.A0, D.A1, D.axis, item - D.slot0, miss, bad);
        if (bad) atomicAdd(&D.err[ERR_WALK], bad);
        if (miss) atomicAdd(&D.err[ERR_TEMPLATE], miss);
    }
    // segment counts per mesh: lanes of a warp that share a descriptor add once
    const unsigned group = __match_any_sync(0xffffffffu, d);
    const unsigned sum = __reduce_add_sync(group, (unsigned)nseg);
    if ((threadIdx.x & 31) == __ffs(group) - 1 && sum && item - (threadIdx.x & 31) < n_items)
        atomicAdd(descs[d].seg, (unsigned long long)sum);
}

// tables of the table-driven power for each descriptor (grid: descriptor x 8 entries,
// 256 cells)
__global__ void k_pow_tables_batch(const WalkDesc *__restrict__ descs) {
    const WalkDesc &D = descs[blockIdx.x];
    fill_pow_entry(D.A0.p_exp, threadIdx.x, blockIdx.y, const_cast<float2 *>(D.A0.pow_cell),
                   const_cast<float2 *>(D.A0.pow_exp));
}

// Path export: same walk, segments written out for requested lines.
__global__ void k_walk_paths(WalkGeom W, int axis, int dir, const int64_t *__restrict__ gps,
                             int64_t n_lines, int64_t n_gp, int cap, int32_t *tet_out, double *r0_out,
                             double *r1_out, int32_t *nseg_out) {
    int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= n_lines) return;
    int64_t g = gps[l];
    if (g < 0 || g >= n_gp) {
        nseg_out[l] = -1;
        return;
    }
    const double x0 = W.gp[3 * g], x1 = W.gp[3 * g + 1], x2 = W.gp[3 * g + 2];
    const LineF X = line_f(x0, x1, x2, axis);
    int32_t t = (int32_t)(g >> 2);
    double r_prev = 0.0;
    int nseg = 0;
    bool ok = false;
    for (int step = 0; step < W.max_steps; step++) {
        int zmask;
        const double rmax = exit_step(W, X, t, axis, dir, x0, x1, x2, zmask);
        if (!below_inf(rmax)) break;
        if (rmax - r_prev > W.eps_r) {
            if (nseg >= cap) break;
            tet_out[l * cap + nseg] = t;
            r0_out[l * cap + nseg] = r_prev;
            r1_out[l * cap + nseg] = rmax;
            nseg++;
            r_prev = rmax;
        }
        int32_t nx = next_tet(W, t, axis, dir, x0, x1, x2, zmask, rmax);
        if (nx == -1) { ok = true; break; }
        if (nx < 0) break;
        t = nx;
    }
    nseg_out[l] = ok ? nseg : -1;
}

// Gather rows of a binned table into dense rows [n][n_dof] (zero elsewhere).
__global__ void k_table_rows(const float2 *__restrict__ tab, const int32_t *__restrict__ gbin_slot,
                             const int64_t *__restrict__ gps, int64_t n,
                             const int32_t *__restrict__ slot_of_gp,
                             const int32_t *__restrict__ gp_off, const int32_t *__restrict__ dof_off,
                             const int32_t *__restrict__ dof_idx,
                             const int64_t *__restrict__ tab_off, const int32_t *__restrict__ tab_ld,
                             int64_t n_dof, int64_t n_gp, double *rows) {
    int64_t l = blockIdx.x;
    if (l >= n) return;
    int64_t g = gps[l];
    if (g < 0 || g >= n_gp) return;
    int32_t slot = slot_of_gp[g];
    int32_t bin = gbin_slot[slot];
    int32_t row = slot - gp_off[bin];
    int d0 = dof_off[bin], nd = dof_off[bin + 1] - d0;
    for (int c = threadIdx.x; c < nd; c += blockDim.x) {
        const float2 v = tab[tab_off[bin] + (int64_t)c * tab_ld[bin] + row];
        rows[l * n_dof + dof_idx[d0 + c]] = (double)v.x + (double)v.y;
    }
}

WalkGeom make_geom(Mesh *m) {
    WalkGeom W;
    W.M = m->M; W.inv = m->inv; W.rec = m->recf; W.tets = m->tets; W.nbr = m->nbr; W.dof = m->dof;
    W.vt_off = m->vt_off; W.vt_tet = m->vt_tet; W.gp = m->gp;
    W.eps_r = kEpsRRel * m->span;
    W.max_steps = m->max_steps;
    return W;
}

}  // namespace

int walk_tables(Mesh *m, const double alpha[3]) {
    cudaStream_t s = m->stream;
    WalkGeom W = make_geom(m);
    unsigned long long *segc = reinterpret_cast<unsigned long long *>(m->norms + kSegCounterSlot);
    FEM3_CUDA(cudaMemsetAsync(segc, 0, sizeof(unsigned long long), s));
    if (!m->pow_cell) {
        FEM3_TRY(dev_alloc_t(m, &m->pow_cell, 3 * 256 * 8));
        FEM3_TRY(dev_alloc_t(m, &m->pow_exp, 3 * 128));
    }
    k_pow_tables<<<dim3(8, 3), 256, 0, s>>>(1.0 - alpha[0] / 2.0, 1.0 - alpha[1] / 2.0,
                                            1.0 - alpha[2] / 2.0, m->pow_cell, m->pow_exp);
    note_launch(m);
    stage_begin(m, 2);
    AxisTables T;
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        double gamma = alpha[axis] / 2.0;
        double ig = 1.0 / tgamma(2.0 - gamma);
        const float igh = (float)ig, igl = (float)(ig - (double)igh);
        T.A0[axis] = TableArgs{B.gp_idx, B.slot_bin, B.gp_off, B.dof_off, B.dof_key, B.dof_q,
                               B.tab_off, B.tab_ld, m->tabL[axis], 1.0 - gamma, igh, igl,
                               m->pow_cell + (size_t)axis * 256 * 8, m->pow_exp + axis * 128};
        T.A1[axis] = T.A0[axis];
        T.A1[axis].tab = m->tabR[axis];
        T.A1[axis].coef_h = -igh;
        T.A1[axis].coef_l = -igl;
    }
    // one line per lane (128 slots a block) up to eight blocks per SM and axis; beyond that
    // the blocks hold more slots and their lanes take further lines as they finish.  (At the
    // 16^3 cube 2.5 lines per lane was 10 % slower than one: the lanes of a warp drift to
    // different lines and diverge.)
    // the slots of this part's bins (all slots unless the mesh is assembled in parts)
    int64_t span = 0;
    for (int axis = 0; axis < 3; axis++) {
        int b0, b1;
        part_bins(m, axis, b0, b1);
        T.lo[axis] = m->bins[axis].h_gp_off[b0];
        T.hi[axis] = m->bins[axis].h_gp_off[b1];
        span = std::max(span, T.hi[axis] - T.lo[axis]);
    }
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        FEM3_CUDA(cudaGetDevice(&dev));
        FEM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int64_t blocks = std::max<int64_t>(1, (int64_t)sms * 8);
    const int per_block = (int)std::max<int64_t>(128, (span + blocks - 1) / blocks);
    kc_begin(m, KC_WALK);
    k_walk_tables<<<dim3((unsigned)std::max<int64_t>(1, (span + per_block - 1) / per_block), 3),
                    128, 0, s>>>(W, T, m->n_gp, per_block, 0, m->err, segc);
    kc_end(m, KC_WALK);
    note_launch(m);
    stage_end(m, 2);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// Tables of one axis for the general form (c D^a u, D^^b v) (Section 2.1, eq. "equ:varsss"):
// the left table L with order order_left and the right table R with order order_right, each
// in [0, 1] (order 0: the basis function itself; order 1: the slope on the Gauss point's
// tet), both with the one-sided coefficient +-1/Gamma(2 - order).  The power tables of
// slots 0 and 1 take the two exponents.
int walk_tables_form(Mesh *m, int axis, double order_left, double order_right) {
    cudaStream_t s = m->stream;
    WalkGeom W = make_geom(m);
    unsigned long long *segc = reinterpret_cast<unsigned long long *>(m->norms + kSegCounterSlot);
    FEM3_CUDA(cudaMemsetAsync(segc, 0, sizeof(unsigned long long), s));
    if (!m->pow_cell) {
        FEM3_TRY(dev_alloc_t(m, &m->pow_cell, 3 * 256 * 8));
        FEM3_TRY(dev_alloc_t(m, &m->pow_exp, 3 * 128));
    }
    k_pow_tables<<<dim3(8, 3), 256, 0, s>>>(1.0 - order_left, 1.0 - order_right,
                                            1.0 - order_right, m->pow_cell, m->pow_exp);
    note_launch(m);
    AxisBins &B = m->bins[axis];
    AxisTables T;
    const double il = 1.0 / tgamma(2.0 - order_left), ir = 1.0 / tgamma(2.0 - order_right);
    const float ilh = (float)il, ill = (float)(il - (double)ilh);
    const float irh = (float)ir, irl = (float)(ir - (double)irh);
    T.A0[axis] = TableArgs{B.gp_idx, B.slot_bin, B.gp_off, B.dof_off, B.dof_key, B.dof_q,
                           B.tab_off, B.tab_ld, m->tabL[axis], 1.0 - order_left, ilh, ill,
                           m->pow_cell, m->pow_exp};
    T.A1[axis] = TableArgs{B.gp_idx, B.slot_bin, B.gp_off, B.dof_off, B.dof_key, B.dof_q,
                           B.tab_off, B.tab_ld, m->tabR[axis], 1.0 - order_right, -irh, -irl,
                           m->pow_cell + 256 * 8, m->pow_exp + 128};
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        FEM3_CUDA(cudaGetDevice(&dev));
        FEM3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int64_t blocks = std::max<int64_t>(1, (int64_t)sms * 8);
    const int per_block = (int)std::max<int64_t>(128, (m->n_gp + blocks - 1) / blocks);
    T.lo[axis] = 0;
    T.hi[axis] = m->n_gp;
    kc_begin(m, KC_WALK);
    k_walk_tables<<<dim3((unsigned)((m->n_gp + per_block - 1) / per_block), 1), 128, 0, s>>>(
        W, T, m->n_gp, per_block, axis, m->err, segc);
    kc_end(m, KC_WALK);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int walk_paths(Mesh *m, int axis, int dir, const int64_t *gps, int64_t n, int cap,
               int32_t *tet_out, double *r0, double *r1, int32_t *nseg) {
    WalkGeom W = make_geom(m);
    k_walk_paths<<<(unsigned)((n + 127) / 128), 128, 0, m->stream>>>(W, axis, dir, gps, n, m->n_gp,
                                                                      cap, tet_out, r0, r1, nseg);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int table_rows(Mesh *m, int axis, int dir, const int64_t *gps, int64_t n, double *rows) {
    cudaStream_t s = m->stream;
    AxisBins &B = m->bins[axis];
    const int32_t *slot_of_gp = B.slot_of_gp;
    FEM3_CUDA(cudaMemsetAsync(rows, 0, sizeof(double) * n * m->n_dof, s));
    const float2 *tab = dir < 0 ? m->tabL[axis] : m->tabR[axis];
    if (n > 0) {
        k_table_rows<<<(unsigned)n, 128, 0, s>>>(tab, B.slot_bin, gps, n, slot_of_gp, B.gp_off,
                                                  B.dof_off, B.dof_idx, B.tab_off, B.tab_ld,
                                                  m->n_dof, m->n_gp, rows);
        note_launch(m);
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

// Walk + tables for every mesh of a batch in two launches (power tables, walk; the walk
// zeroes each line's table rows itself).  Scratch: a device and a pinned host descriptor
// array owned by the caller, sized for the batch.
int walk_tables_batch(Mesh *const *ms, int n, const double *alpha, cudaStream_t s,
                      BatchWalkScratch *bs) {
    const int n_desc = 3 * n;
    if (!bs->d_desc) {
        FEM3_CUDA(cudaMalloc(&bs->d_desc, sizeof(WalkDesc) * n_desc));
        FEM3_CUDA(cudaMallocHost(&bs->h_desc, sizeof(WalkDesc) * n_desc));
    }
    WalkDesc *hd = reinterpret_cast<WalkDesc *>(bs->h_desc);
    int64_t items = 0;
    for (int i = 0; i < n; i++) {
        Mesh *m = ms[i];
        if (!m->pow_cell) {
            FEM3_TRY(dev_alloc_t(m, &m->pow_cell, 3 * 256 * 8));
            FEM3_TRY(dev_alloc_t(m, &m->pow_exp, 3 * 128));
        }
        WalkGeom W = make_geom(m);
        for (int axis = 0; axis < 3; axis++) {
            AxisBins &B = m->bins[axis];
            const double gamma = alpha[3 * i + axis] / 2.0;
            const double ig = 1.0 / tgamma(2.0 - gamma);
            const float igh = (float)ig, igl = (float)(ig - (double)igh);
            WalkDesc &D = hd[3 * i + axis];
            D.W = W;
            D.A0 = TableArgs{B.gp_idx, B.slot_bin, B.gp_off, B.dof_off, B.dof_key, B.dof_q,
                             B.tab_off, B.tab_ld, m->tabL[axis], 1.0 - gamma, igh, igl,
                             m->pow_cell + (size_t)axis * 256 * 8, m->pow_exp + axis * 128};
            D.A1 = D.A0;
            D.A1.tab = m->tabR[axis];
            D.A1.coef_h = -igh;
            D.A1.coef_l = -igl;
            D.axis = axis;
            D.slot0 = items;
            D.n_gp = m->n_gp;
            D.err = m->err;
            D.seg = reinterpret_cast<unsigned long long *>(m->norms + kSegCounterSlot);
            items += m->n_gp;
        }
        FEM3_CUDA(cudaMemsetAsync(m->norms + kSegCounterSlot, 0, sizeof(double), s));
    }
    FEM3_CUDA(cudaMemcpyAsync(bs->d_desc, hd, sizeof(WalkDesc) * n_desc, cudaMemcpyHostToDevice, s));
    k_pow_tables_batch<<<dim3(n_desc, 8), 256, 0, s>>>(
        reinterpret_cast<const WalkDesc *>(bs->d_desc));
    if (items > 0)
        k_walk_batch<<<(unsigned)((items + 127) / 128), 128, 0, s>>>(
            reinterpret_cast<const WalkDesc *>(bs->d_desc), n_desc, items);
    for (int i = 0; i < n; i++) ms[i]->launches += 2;   // the batch's launches, counted per mesh
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

}  // namespace fem3
