// Mesh records on the device (Section 2.2 volume coordinates and adjacency, Section 2.1
// Gauss rule, Section 2.3 template sets per transverse bin).
#include <math.h>

#include <algorithm>
#include <cstring>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

constexpr int kThreads = 256;
constexpr unsigned long long kEmptyKey = ~0ull;

inline unsigned grid_for(int64_t n, int threads = kThreads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);   // kernels check their bounds; never a 0-size grid
}

// order-preserving map of a double to an unsigned 64-bit integer (for atomic min/max)
__device__ __forceinline__ unsigned long long ord_of(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double double_of_ord(unsigned long long o) {
    unsigned long long b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
    return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------------------------
// per tet: barycentric map, gradient reciprocals, volume, Gauss points, bounding box
// ---------------------------------------------------------------------------------
__global__ void k_tet_geom(const double *__restrict__ verts, const int32_t *__restrict__ tets,
                           int64_t n_tets, int64_t n_nodes, double qa, double qb,
                           double *__restrict__ M, double *__restrict__ inv,
                           float4 *__restrict__ recf, double *__restrict__ vol,
                           double *__restrict__ gp, double *__restrict__ gw,
                           unsigned long long *__restrict__ node_box, int32_t *__restrict__ err) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_tets) return;
    double v[4][3];
    for (int k = 0; k < 4; k++) {
        int32_t id = tets[4 * t + k];
        if (id < 0 || id >= n_nodes) {
            atomicAdd(&err[ERR_MESH], 1);
            return;
        }
        for (int d = 0; d < 3; d++) v[k][d] = verts[3 * id + d];
    }
    // edge vectors e_c = v_{c+1} - v_0 and det (no contraction: same rounding as a plain
    // evaluation of the triple product, so the weights match any IEEE evaluation)
    double e[3][3];
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) e[c][d] = __dsub_rn(v[c + 1][d], v[0][d]);
    double m0 = __dsub_rn(__dmul_rn(e[1][1], e[2][2]), __dmul_rn(e[1][2], e[2][1]));
    double m1 = __dsub_rn(__dmul_rn(e[1][0], e[2][2]), __dmul_rn(e[1][2], e[2][0]));
    double m2 = __dsub_rn(__dmul_rn(e[1][0], e[2][1]), __dmul_rn(e[1][1], e[2][0]));
    double det = __dadd_rn(__dsub_rn(__dmul_rn(e[0][0], m0), __dmul_rn(e[0][1], m1)),
                           __dmul_rn(e[0][2], m2));
    double emax = 0;
    for (int c = 0; c < 3; c++)
        for (int d = 0; d < 3; d++) emax = fmax(emax, fabs(e[c][d]));
    if (!(fabs(det) > 1e-14 * emax * emax * emax)) {
        atomicAdd(&err[ERR_MESH], 1);
        return;
    }
    double V = __ddiv_rn(fabs(det), 6.0);
    vol[t] = V;
    // gradients of lambda_1..3 are the rows of J^{-1}, J = [e_0 e_1 e_2] (columns):
    // grad lambda_1 = (e_1 x e_2)/det, grad lambda_2 = (e_2 x e_0)/det,
    // grad lambda_3 = (e_0 x e_1)/det
    double g[4][3];
    const int pa[3] = {1, 2, 0}, pb[3] = {2, 0, 1};
    double rdet = 1.0 / det;
    for (int r = 0; r < 3; r++) {
        const double *a = e[pa[r]], *b = e[pb[r]];
        g[r + 1][0] = (a[1] * b[2] - a[2] * b[1]) * rdet;
        g[r + 1][1] = (a[2] * b[0] - a[0] * b[2]) * rdet;
        g[r + 1][2] = (a[0] * b[1] - a[1] * b[0]) * rdet;
    }
    for (int d = 0; d < 3; d++) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    double c[4];
    c[1] = -(g[1][0] * v[0][0] + g[1][1] * v[0][1] + g[1][2] * v[0][2]);
    c[2] = -(g[2][0] * v[0][0] + g[2][1] * v[0][1] + g[2][2] * v[0][2]);
    c[3] = -(g[3][0] * v[0][0] + g[3][1] * v[0][1] + g[3][2] * v[0][2]);
    c[0] = 1.0 - (c[1] + c[2] + c[3]);
    double *Mt = M + 16 * t;
    for (int k = 0; k < 4; k++) {
        Mt[4 * k + 0] = c[k];
        Mt[4 * k + 1] = g[k][0];
        Mt[4 * k + 2] = g[k][1];
        Mt[4 * k + 3] = g[k][2];
    }
    double iv[3][4];
    for (int a = 0; a < 3; a++) {
        double ds = 0;
        for (int k = 0; k < 4; k++) ds = fmax(ds, fabs(g[k][a]));
        for (int k = 0; k < 4; k++) {
            iv[a][k] = fabs(g[k][a]) > kEpsDRel * ds ? 1.0 / g[k][a] : 0.0;
            inv[12 * t + 4 * a + k] = iv[a][k];
        }
    }
    // FP32 records of the walk's exit filter, one 128-byte record per (tet, axis), in
    // tet-local form lambda_k(x) = A_k + grad lambda_k . (x - c_T) about an FP32 point c_T
    // (the rounded centroid):
    //   [0] A_k = lambda_k(c_T); [1], [2] hi + lo split of dlambda_k/dx_axis (the table
    //   factor); [3] FP32 copy of the FP64 reciprocal (same sign, 0 where it is 0);
    //   [4], [5] dlambda_k/dx_p1, dlambda_k/dx_p2 for p1 = axis + 1, p2 = axis + 2 (mod 3);
    //   [6] (c_p1, c_p2, F0, Gmax): Gmax >= max_k sum_i |dlambda_k/dx_i| and
    //   F0 >= 1 + Gmax |c_T|_inf, both rounded up; [7] unused.
    // The filter that reads them decides only what its error bounds separate (the FP64
    // step decides the rest).
    float cT[3];
    for (int d = 0; d < 3; d++)
        cT[d] = __double2float_rn(0.25 * (((v[0][d] + v[1][d]) + v[2][d]) + v[3][d]));
    float Ak[4];
    double gs = 0.0, cn = 0.0;
    for (int k = 0; k < 4; k++) {
        Ak[k] = __double2float_rn(c[k] + g[k][0] * (double)cT[0] + g[k][1] * (double)cT[1] +
                                  g[k][2] * (double)cT[2]);
        gs = fmax(gs, fabs(g[k][0]) + fabs(g[k][1]) + fabs(g[k][2]));
    }
    for (int d = 0; d < 3; d++) cn = fmax(cn, fabs((double)cT[d]));
    // values far outside FP32's normal range make the filter defer every step (F0 = inf)
    bool in_range = gs * cn < 0x1p100;
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < 4; k++) {
            const double ga = fabs(g[k][a]), ia = fabs(iv[a][k]);
            in_range &= (ga == 0.0 || (ga > 0x1p-100 && ga < 0x1p100)) &&
                        (ia == 0.0 || (ia > 0x1p-100 && ia < 0x1p100));
        }
    const float gmax = __double2float_ru(gs * (1.0 + 1e-9));
    const float f0 = in_range ? __double2float_ru((1.0 + gs * cn) * (1.0 + 1e-9)) : INFINITY;
    for (int a = 0; a < 3; a++) {
        const int p1 = a == 2 ? 0 : a + 1, p2 = a == 0 ? 2 : a - 1;
        float gh[4], gl[4];
        for (int k = 0; k < 4; k++) f64_split(g[k][a], gh[k], gl[k]);
        float4 *R = recf + 8 * (3 * t + a);
        R[0] = make_float4(Ak[0], Ak[1], Ak[2], Ak[3]);
        R[1] = make_float4(gh[0], gh[1], gh[2], gh[3]);
        R[2] = make_float4(gl[0], gl[1], gl[2], gl[3]);
        R[3] = make_float4(__double2float_rn(iv[a][0]), __double2float_rn(iv[a][1]),
                           __double2float_rn(iv[a][2]), __double2float_rn(iv[a][3]));
        R[4] = make_float4(__double2float_rn(g[0][p1]), __double2float_rn(g[1][p1]),
                           __double2float_rn(g[2][p1]), __double2float_rn(g[3][p1]));
        R[5] = make_float4(__double2float_rn(g[0][p2]), __double2float_rn(g[1][p2]),
                           __double2float_rn(g[2][p2]), __double2float_rn(g[3][p2]));
        R[6] = make_float4(cT[p1], cT[p2], f0, gmax);
        R[7] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // Gauss points: point q has barycentric qa at vertex q, qb elsewhere; summed in
    // vertex order without contraction (bit-identical to a plain IEEE evaluation)
    for (int q = 0; q < 4; q++) {
        for (int d = 0; d < 3; d++) {
            double x = 0.0;
            for (int k = 0; k < 4; k++) x = __dadd_rn(x, __dmul_rn(k == q ? qa : qb, v[k][d]));
            gp[3 * (4 * t + q) + d] = x;
        }
        gw[4 * t + q] = __ddiv_rn(V, 4.0);
    }
    // element-patch bounding boxes of the four vertices
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        lo[d] = fmin(fmin(v[0][d], v[1][d]), fmin(v[2][d], v[3][d]));
        hi[d] = fmax(fmax(v[0][d], v[1][d]), fmax(v[2][d], v[3][d]));
    }
    for (int k = 0; k < 4; k++) {
        int32_t id = tets[4 * t + k];
        for (int d = 0; d < 3; d++) {
            atomicMin(&node_box[6 * (int64_t)id + d], ord_of(lo[d]));
            atomicMax(&node_box[6 * (int64_t)id + 3 + d], ord_of(hi[d]));
        }
    }
}

// bounding box of the vertices (ordered-integer atomics) and total volume
// bounding box of the nodes and total tet volume: reduced within each warp first, one
// atomic per warp and quantity
// The volume goes into one partial sum per warp (no atomics) and k_sum_ordered adds the
// partials in a fixed order: the total, and the bin width derived from it, are the same
// bits on every run (with atomics the order of the additions varied, the last bit of the
// width with it, and at a width that divides the extent the bin count flipped).
__global__ void k_extent(const double *__restrict__ verts, int64_t n_nodes,
                         const double *__restrict__ vol, int64_t n_tets,
                         unsigned long long *ext, double *vpart) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        unsigned long long lo = ~0ull, hi = 0ull;
        if (i < n_nodes) lo = hi = ord_of(verts[3 * i + d]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o);
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, hi, o);
            lo = a < lo ? a : lo;
            hi = b > hi ? b : hi;
        }
        if (lane == 0 && lo != ~0ull) {
            atomicMin(&ext[d], lo);
            atomicMax(&ext[3 + d], hi);
        }
    }
    double v = i < n_tets ? vol[i] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) vpart[i >> 5] = v;
}

// out = sum of in[0 .. n) in a fixed order (one block of 256 threads)
__global__ void k_sum_ordered(const double *__restrict__ in, int64_t n, double *out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 256) a += in[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_box_init(unsigned long long *box, int64_t n_nodes) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 6 * n_nodes) return;
    box[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

__global__ void k_box_decode(unsigned long long *box, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = double_of_ord(box[i]);
    reinterpret_cast<double *>(box)[i] = v;
}

// ---------------------------------------------------------------------------------
// face neighbours by hashing sorted vertex triples
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long face_key(const int32_t *tv, int k) {
    int32_t f[3];
    int n = 0;
    for (int q = 0; q < 4; q++)
        if (q != k) f[n++] = tv[q];
    if (f[1] < f[0]) { int32_t s = f[0]; f[0] = f[1]; f[1] = s; }
    if (f[2] < f[1]) { int32_t s = f[1]; f[1] = f[2]; f[2] = s; }
    if (f[1] < f[0]) { int32_t s = f[0]; f[0] = f[1]; f[1] = s; }
    return ((unsigned long long)f[0] << 42) | ((unsigned long long)f[1] << 21) |
           (unsigned long long)f[2];
}

__device__ __forceinline__ unsigned long long hash_slot(unsigned long long key, int bits) {
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - bits);
}

__global__ void k_face_insert(const int32_t *__restrict__ tets, int64_t n_tets,
                              unsigned long long *keys, int32_t *vals, int bits,
                              int32_t *err) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * n_tets) return;
    int64_t t = f >> 2;
    int k = (int)(f & 3);
    unsigned long long key = face_key(tets + 4 * t, k);
    unsigned long long mask = (1ull << bits) - 1;
    unsigned long long h = hash_slot(key, bits);
    for (int probe = 0; probe < 4096; probe++) {
        unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) {
            if (atomicCAS(&vals[2 * h], -1, (int32_t)f) != -1 &&
                atomicCAS(&vals[2 * h + 1], -1, (int32_t)f) != -1)
                atomicAdd(&err[ERR_FACE], 1);  // face shared by more than two tets
            return;
        }
        h = (h + 1) & mask;
    }
    atomicAdd(&err[ERR_FACE], 1);
}

__global__ void k_face_match(const int32_t *__restrict__ tets, int64_t n_tets,
                             const unsigned long long *__restrict__ keys,
                             const int32_t *__restrict__ vals, int bits,
                             int32_t *__restrict__ nbr, int32_t *err) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * n_tets) return;
    int64_t t = f >> 2;
    int k = (int)(f & 3);
    unsigned long long key = face_key(tets + 4 * t, k);
    unsigned long long mask = (1ull << bits) - 1;
    unsigned long long h = hash_slot(key, bits);
    for (int probe = 0; probe < 4096; probe++) {
        if (keys[h] == key) {
            int32_t a = vals[2 * h], b = vals[2 * h + 1];
            int32_t other = (a == (int32_t)f) ? b : a;
            nbr[f] = other >= 0 ? (other >> 2) : -1;
            return;
        }
        h = (h + 1) & mask;
    }
    nbr[f] = -1;
    atomicAdd(&err[ERR_FACE], 1);
}

__global__ void k_mark_nodes(const int32_t *__restrict__ tets, const int32_t *__restrict__ nbr,
                             int64_t n_tets, int64_t n_nodes, int32_t *used, int32_t *bnd,
                             int32_t *vt_count) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * n_tets) return;
    int64_t t = f >> 2;
    int k = (int)(f & 3);
    for (int q = 0; q < 4; q++) {
        int32_t id = tets[4 * t + q];
        if (id < 0 || id >= n_nodes) return;   // reported by k_tet_geom
    }
    int32_t node = tets[f];
    used[node] = 1;
    atomicAdd(&vt_count[node], 1);
    if (nbr[f] < 0)
        for (int q = 0; q < 4; q++)
            if (q != k) bnd[tets[4 * t + q]] = 1;
}

__global__ void k_interior_flag(const int32_t *used, const int32_t *bnd, int64_t n,
                                int32_t *flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (used[i] && !bnd[i]) ? 1 : 0;
}

__global__ void k_dof_number(const int32_t *flag, const int32_t *off, int64_t n,
                             int32_t *dof, int32_t *dof_node) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (flag[i]) {
        dof[i] = off[i];
        dof_node[off[i]] = (int32_t)i;
    } else {
        dof[i] = -1;
    }
}

__global__ void k_vt_fill(const int32_t *__restrict__ tets, int64_t n_tets, int64_t n_nodes,
                          const int32_t *__restrict__ off, int32_t *cursor, int32_t *vt_tet) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * n_tets) return;
    int32_t node = tets[f];
    if (node < 0 || node >= n_nodes) return;
    int32_t pos = atomicAdd(&cursor[node], 1);
    vt_tet[off[node] + pos] = (int32_t)(f >> 2);
}

// ---------------------------------------------------------------------------------
// scan (three-phase: per-block sums, scan of block sums, add back)
// ---------------------------------------------------------------------------------
constexpr int kScanBlock = 1024;

__device__ int32_t block_excl_scan(int32_t v, int32_t *sh, int32_t *total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int32_t base = w > 0 ? sh[w - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void k_scan_blocks(const int32_t *in, int32_t *out, int64_t n, int32_t *bsum) {
    __shared__ int32_t sh[32];
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    int32_t v = i < n ? in[i] : 0, tot;
    int32_t e = block_excl_scan(v, sh, &tot);
    if (i < n) out[i] = e;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *bsum, int64_t nb, int32_t *total_out) {
    __shared__ int32_t sh[32];
    int32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        int64_t i = base + threadIdx.x;
        int32_t v = i < nb ? bsum[i] : 0, tot;
        int32_t e = block_excl_scan(v, sh, &tot);
        if (i < nb) bsum[i] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *bsum) {
    int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// ---------------------------------------------------------------------------------
// transverse bins of one axis
// ---------------------------------------------------------------------------------
struct BinGeom {
    int c0, c1, nb0, nb1;
    double org0, org1, width;
};

__device__ __forceinline__ int bin_coord(double p, double org, double w, int nb) {
    double q = floor((p - org) / w);
    int i = q < 0 ? 0 : (q > nb - 1 ? nb - 1 : (int)q);
    return i;
}

// ---------------------------------------------------------------------------------
// Transverse bins of the three axes, built together: one launch per step with
// blockIdx.y = axis.
// ---------------------------------------------------------------------------------
struct BinAxis {
    BinGeom G;
    int32_t *gcount, *dcount, *gcur, *dcur, *gbin, *gp_off, *dof_off;
    unsigned long long *gkeys, *dkeys;
    int32_t *gp_idx, *slot_bin, *dof_idx, *row_bin, *slot_of_gp;
    uint32_t *dq;   // [n_dof] quantised position of each dof's element patch along the axis
    double *w_slot;
    double lo, span;   // extent along the axis (sort key of the Gauss points)
    int n_bins;
};
struct BinAxes {
    BinAxis a[3];
};

__global__ void k_bin_count3(const __grid_constant__ BinAxes P, const double *__restrict__ gp,
                             int64_t n_gp, const double *__restrict__ box,
                             const int32_t *__restrict__ dof_node, int64_t n_dof) {
    const BinAxis &X = P.a[blockIdx.y];
    const BinGeom G = X.G;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_gp) {
        const int i0 = bin_coord(gp[3 * i + G.c0], G.org0, G.width, G.nb0);
        const int i1 = bin_coord(gp[3 * i + G.c1], G.org1, G.width, G.nb1);
        const int b = i0 + G.nb0 * i1;
        X.gbin[i] = b;
        // lanes of a warp (neighbouring Gauss points) mostly share a bin: one atomic per bin
        const unsigned grp = __match_any_sync(__activemask(), b);
        if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&X.gcount[b], __popc(grp));
    }
    if (i < n_dof) {
        const double *bx = box + 6 * (int64_t)dof_node[i];
        const int a0 = bin_coord(bx[G.c0], G.org0, G.width, G.nb0);
        const int a1 = bin_coord(bx[3 + G.c0], G.org0, G.width, G.nb0);
        const int b0 = bin_coord(bx[G.c1], G.org1, G.width, G.nb1);
        const int b1 = bin_coord(bx[3 + G.c1], G.org1, G.width, G.nb1);
        for (int i1 = b0; i1 <= b1; i1++)
            for (int i0 = a0; i0 <= a1; i0++) atomicAdd(&X.dcount[i0 + G.nb0 * i1], 1);
    }
}

// exclusive scans of the six count arrays (block q: axis q / 2, Gauss points or dofs),
// total in out[n]; one CTA per array
__global__ void k_bin_scan3(const __grid_constant__ BinAxes P) {
    __shared__ int32_t sh[32];
    const BinAxis &X = P.a[blockIdx.x >> 1];
    const bool dofs = blockIdx.x & 1;
    const int32_t *in = dofs ? X.dcount : X.gcount;
    int32_t *out = dofs ? X.dof_off : X.gp_off;
    const int n = X.n_bins;
    int32_t carry = 0;
    for (int base = 0; base < n; base += kScanBlock) {
        const int i = base + threadIdx.x;
        int32_t v = i < n ? in[i] : 0, tot;
        const int32_t e = block_excl_scan(v, sh, &tot);
        if (i < n) out[i] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_bin_fill3(const __grid_constant__ BinAxes P, const double *__restrict__ gp,
                            int64_t n_gp, const double *__restrict__ box,
                            const int32_t *__restrict__ dof_node, int64_t n_dof) {
    const int axis = blockIdx.y;
    const BinAxis &X = P.a[axis];
    const BinGeom G = X.G;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_gp) {
        const int b = X.gbin[i];
        // one atomic per bin and warp; lanes take consecutive places (the bin is sorted later)
        const unsigned grp = __match_any_sync(__activemask(), b);
        const int lead = __ffs(grp) - 1, lane = threadIdx.x & 31;
        int32_t base = 0;
        if (lane == lead) base = atomicAdd(&X.gcur[b], __popc(grp));
        const int32_t pos = __shfl_sync(grp, base, lead) + __popc(grp & ((1u << lane) - 1u));
        // sort key: position along the axis (30-bit quantised), then the Gauss point id
        double u = (gp[3 * i + axis] - X.lo) / X.span;
        u = u < 0 ? 0 : (u > 1 ? 1 : u);
        const unsigned long long q = (unsigned long long)(u * 1073741823.0);
        X.gkeys[X.gp_off[b] + pos] = (q << 32) | (unsigned long long)i;
    }
    if (i < n_dof) {
        const double *bx = box + 6 * (int64_t)dof_node[i];
        const int a0 = bin_coord(bx[G.c0], G.org0, G.width, G.nb0);
        const int a1 = bin_coord(bx[3 + G.c0], G.org0, G.width, G.nb0);
        const int b0 = bin_coord(bx[G.c1], G.org1, G.width, G.nb1);
        const int b1 = bin_coord(bx[3 + G.c1], G.org1, G.width, G.nb1);
        // sort key of a template row: the lower end of the dof's element patch along the
        // axis (30-bit quantised), then the dof id.  With the Gauss points of a bin sorted
        // along the axis as well, a row's nonzeros in the left table (paths running from the
        // Gauss point towards -x) start at a Gauss point that grows with the key, and those
        // in the right table end at one: the apply skips the rest of each row.
        double u = (bx[axis] - X.lo) / X.span;
        u = u < 0 ? 0 : (u > 1 ? 1 : u);
        const uint32_t q = (uint32_t)(u * 1073741823.0);
        X.dq[i] = q;
        const unsigned long long key = ((unsigned long long)q << 32) | (unsigned long long)i;
        for (int i1 = b0; i1 <= b1; i1++)
            for (int i0 = a0; i0 <= a1; i0++) {
                const int b = i0 + G.nb0 * i1;
                const int32_t pos = atomicAdd(&X.dcur[b], 1);
                X.dkeys[X.dof_off[b] + pos] = key;
            }
    }
}

// one CTA per (bin, axis, kind): bitonic sort of the bin's keys in shared memory (sized by
// the launch for the largest bin, rounded up to a power of two); kind 0 writes the
// Gauss-point ids and the slot -> bin map, kind 1 the dof ids and the row -> bin map
__global__ void k_bin_sort3(const __grid_constant__ BinAxes P) {
    extern __shared__ unsigned long long sh[];
    const BinAxis &X = P.a[blockIdx.y];
    const int b = blockIdx.x;
    if (b >= X.n_bins) return;
    const bool dofs = blockIdx.z == 1;
    const int32_t *off = dofs ? X.dof_off : X.gp_off;
    const unsigned long long *keys = dofs ? X.dkeys : X.gkeys;
    int32_t *ids = dofs ? X.dof_idx : X.gp_idx;
    int32_t *bin_of = dofs ? X.row_bin : X.slot_bin;
    const int lo = off[b], n = off[b + 1] - lo;
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int i = threadIdx.x; i < p2; i += blockDim.x) sh[i] = i < n ? keys[lo + i] : ~0ull;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = sh[i], c = sh[l];
                    if ((a > c) == up) { sh[i] = c; sh[l] = a; }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        ids[lo + i] = (int32_t)(sh[i] & 0xffffffffull);
        bin_of[lo + i] = b;
        if (dofs) X.dkeys[lo + i] = sh[i];   // the walk searches a row by its key
    }
}

// slot weights and the Gauss point -> slot map of each axis
__global__ void k_bin_slots3(const __grid_constant__ BinAxes P, const double *__restrict__ gw,
                             int64_t n_gp) {
    const BinAxis &X = P.a[blockIdx.y];
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n_gp) return;
    const int32_t g = X.gp_idx[s];
    X.w_slot[s] = gw[g];
    X.slot_of_gp[g] = (int32_t)s;
}

}  // namespace

// ---------------------------------------------------------------------------------
int scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, Mesh *m) {
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb < 1) nb = 1;
    int32_t *bsum = nullptr;
    FEM3_TRY(dev_alloc_t(m, &bsum, nb));
    k_scan_blocks<<<(unsigned)nb, kScanBlock, 0, s>>>(in, out, n, bsum);
    note_launch(m);
    k_scan_sums<<<1, kScanBlock, 0, s>>>(bsum, nb, out + n);
    note_launch(m);
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, s>>>(out, n, bsum);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int mesh_build(Mesh *m, const double *verts_d, const int32_t *tets_d) {
    cudaStream_t s = m->stream;
    const int64_t T = m->n_tets, N = m->n_nodes;
    FEM3_TRY(dev_alloc_t(m, &m->M, 16 * T));
    FEM3_TRY(dev_alloc_t(m, &m->inv, 12 * T));
    FEM3_TRY(dev_alloc_t(m, &m->recf, 24 * T));
    FEM3_TRY(dev_alloc_t(m, &m->vol, T));
    FEM3_TRY(dev_alloc_t(m, &m->nbr, 4 * T));
    FEM3_TRY(dev_alloc_t(m, &m->dof, N));
    FEM3_TRY(dev_alloc_t(m, &m->vt_off, N + 1));
    FEM3_TRY(dev_alloc_t(m, &m->vt_tet, 4 * T));
    FEM3_TRY(dev_alloc_t(m, &m->gp, 3 * m->n_gp));
    FEM3_TRY(dev_alloc_t(m, &m->gw, m->n_gp));
    FEM3_TRY(dev_alloc_t(m, &m->node_box, 6 * N));

    // Gauss rule constants, evaluated like any IEEE host evaluation of the same formula
    const double qa = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
    const double qb = (5.0 - sqrt(5.0)) / 20.0;

    unsigned long long *box = reinterpret_cast<unsigned long long *>(m->node_box);
    k_box_init<<<grid_for(6 * N), kThreads, 0, s>>>(box, N);
    note_launch(m);
    // 64-thread blocks: one long FP64 thread per tet, spread over every SM
    k_tet_geom<<<grid_for(T, 64), 64, 0, s>>>(verts_d, tets_d, T, N, qa, qb, m->M, m->inv,
                                                 m->recf, m->vol, m->gp, m->gw, box, m->err);
    note_launch(m);
    k_box_decode<<<grid_for(6 * N), kThreads, 0, s>>>(box, 6 * N);
    note_launch(m);

    // face hash: load factor <= 1/4 of 4T face slots
    int bits = 4;
    while ((1ll << bits) < 16 * T) bits++;
    int64_t H = 1ll << bits;
    unsigned long long *keys = nullptr;
    int32_t *vals = nullptr;
    FEM3_TRY(dev_alloc_t(m, &keys, H));
    FEM3_TRY(dev_alloc_t(m, &vals, 2 * H));
    k_fill_u64<<<grid_for(H), kThreads, 0, s>>>(keys, H, kEmptyKey);
    note_launch(m);
    FEM3_CUDA(cudaMemsetAsync(vals, 0xff, sizeof(int32_t) * 2 * H, s));
    k_face_insert<<<grid_for(4 * T), kThreads, 0, s>>>(tets_d, T, keys, vals, bits, m->err);
    note_launch(m);
    k_face_match<<<grid_for(4 * T), kThreads, 0, s>>>(tets_d, T, keys, vals, bits, m->nbr,
                                                       m->err);
    note_launch(m);

    // boundary vertices, dof numbering, vertex -> tets
    int32_t *used, *bnd, *flag, *off, *vcount, *cursor;
    FEM3_TRY(dev_alloc_t(m, &used, N));
    FEM3_TRY(dev_alloc_t(m, &bnd, N));
    FEM3_TRY(dev_alloc_t(m, &flag, N));
    FEM3_TRY(dev_alloc_t(m, &off, N + 1));
    FEM3_TRY(dev_alloc_t(m, &vcount, N));
    FEM3_TRY(dev_alloc_t(m, &cursor, N));
    FEM3_CUDA(cudaMemsetAsync(used, 0, sizeof(int32_t) * N, s));
    FEM3_CUDA(cudaMemsetAsync(bnd, 0, sizeof(int32_t) * N, s));
    FEM3_CUDA(cudaMemsetAsync(vcount, 0, sizeof(int32_t) * N, s));
    FEM3_CUDA(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * N, s));
    k_mark_nodes<<<grid_for(4 * T), kThreads, 0, s>>>(tets_d, m->nbr, T, N, used, bnd, vcount);
    note_launch(m);
    k_interior_flag<<<grid_for(N), kThreads, 0, s>>>(used, bnd, N, flag);
    note_launch(m);
    FEM3_TRY(scan_i32(flag, off, N, s, m));
    FEM3_TRY(scan_i32(vcount, m->vt_off, N, s, m));
    k_vt_fill<<<grid_for(4 * T), kThreads, 0, s>>>(tets_d, T, N, m->vt_off, cursor, m->vt_tet);
    note_launch(m);

    unsigned long long *ext = nullptr;
    double *vsum = nullptr, *vpart = nullptr;
    const unsigned ge = grid_for(std::max(N, T));
    const int64_t nwarp = (int64_t)ge * (kThreads / 32);
    FEM3_TRY(dev_alloc_t(m, &ext, 6));
    FEM3_TRY(dev_alloc_t(m, &vsum, 1));
    FEM3_TRY(dev_alloc_t(m, &vpart, nwarp));
    k_box_init<<<1, 32, 0, s>>>(ext, 1);
    note_launch(m);
    k_extent<<<ge, kThreads, 0, s>>>(verts_d, N, m->vol, T, ext, vpart);
    note_launch(m);
    k_sum_ordered<<<1, 256, 0, s>>>(vpart, nwarp, vsum);
    note_launch(m);

    int32_t n_dof = 0;
    unsigned long long h_ext[6];
    double h_vsum = 0;
    FEM3_CUDA(cudaMemcpyAsync(&n_dof, off + N, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaMemcpyAsync(h_ext, ext, sizeof(h_ext), cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaMemcpyAsync(&h_vsum, vsum, sizeof(double), cudaMemcpyDeviceToHost, s));
    int32_t h_err[ERR_COUNT];
    FEM3_CUDA(cudaMemcpyAsync(h_err, m->err, sizeof(h_err), cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    if (h_err[ERR_MESH]) return set_error(FEM3_E_MESH, "degenerate tetrahedron or node id out of range");
    if (h_err[ERR_FACE]) return set_error(FEM3_E_MESH, "a face is shared by more than two tetrahedra");
    for (int d = 0; d < 6; d++) {
        unsigned long long o = h_ext[d];
        unsigned long long b = (o & 0x8000000000000000ull) ? (o & 0x7fffffffffffffffull) : ~o;
        double v;
        std::memcpy(&v, &b, sizeof(v));
        (d < 3 ? m->lo[d] : m->hi[d - 3]) = v;
    }
    m->span = 0;
    for (int d = 0; d < 3; d++) m->span = std::max(m->span, m->hi[d] - m->lo[d]);
    m->h_est = cbrt(6.0 * h_vsum / (double)T);
    m->n_dof = n_dof;
    FEM3_TRY(dev_alloc_t(m, &m->dof_node, n_dof > 0 ? n_dof : 1));
    k_dof_number<<<grid_for(N), kThreads, 0, s>>>(flag, off, N, m->dof, m->dof_node);
    note_launch(m);
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

int bins_build(Mesh *m) {
    cudaStream_t s = m->stream;
    const int64_t n_gp = m->n_gp, n_dof = m->n_dof;
    // geometry of the three axes' bins; counters and offsets in one allocation each
    BinAxes P;
    int64_t nb_tot = 0;
    int nb_max = 1;
    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        B.c0 = axis == 0 ? 1 : 0;
        B.c1 = axis == 2 ? 1 : 2;
        B.width = m->bin_scale * m->h_est;
        B.org0 = m->lo[B.c0];
        B.org1 = m->lo[B.c1];
        // an extent that is a whole number of widths up to rounding gets that many bins, not
        // one more nearly empty row (points on the far edge clamp into the last bin)
        B.nb0 = std::max(1, (int)ceil((m->hi[B.c0] - m->lo[B.c0]) / B.width * (1.0 - 1e-9)));
        B.nb1 = std::max(1, (int)ceil((m->hi[B.c1] - m->lo[B.c1]) / B.width * (1.0 - 1e-9)));
        B.n_bins = B.nb0 * B.nb1;
        nb_tot += B.n_bins;
        nb_max = std::max(nb_max, B.n_bins);
        BinAxis &X = P.a[axis];
        X = BinAxis{};
        X.G = BinGeom{B.c0, B.c1, B.nb0, B.nb1, B.org0, B.org1, B.width};
        X.lo = m->lo[axis];
        X.span = std::max(m->hi[axis] - m->lo[axis], 1e-300);
        X.n_bins = B.n_bins;
    }
    int32_t *cnt, *offs;
    FEM3_TRY(dev_alloc_t(m, &cnt, 4 * nb_tot));
    FEM3_TRY(dev_alloc_t(m, &offs, 2 * (nb_tot + 3)));
    FEM3_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 4 * nb_tot, s));
    {
        int64_t c = 0, o = 0;
        for (int axis = 0; axis < 3; axis++) {
            AxisBins &B = m->bins[axis];
            BinAxis &X = P.a[axis];
            const int nb = B.n_bins;
            X.gcount = cnt + c;
            X.dcount = cnt + c + nb;
            X.gcur = cnt + c + 2 * nb;
            X.dcur = cnt + c + 3 * nb;
            c += 4 * nb;
            B.gp_off = X.gp_off = offs + o;
            B.dof_off = X.dof_off = offs + o + nb + 1;
            o += 2 * (nb + 1);
            FEM3_TRY(dev_alloc_t(m, &X.gbin, n_gp));
        }
    }
    // pass 1: counts and offsets of all axes, one read-back (device-to-host copies into
    // pageable memory complete before they return)
    const unsigned gx = grid_for(std::max(n_gp, n_dof));
    k_bin_count3<<<dim3(gx, 3), kThreads, 0, s>>>(P, m->gp, n_gp, m->node_box, m->dof_node, n_dof);
    note_launch(m);
    k_bin_scan3<<<6, kScanBlock, 0, s>>>(P);
    note_launch(m);
    std::vector<int32_t> h_offs(2 * (nb_tot + 3));
    FEM3_CUDA(cudaMemcpyAsync(h_offs.data(), offs, sizeof(int32_t) * h_offs.size(),
                              cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    // pass 2: sizes, allocations, then fill, sort and slot maps of all axes in one launch
    // each; host-to-device copies from pageable memory are staged before they return
    int max_gp = 1, max_dof = 1;
    {
        int64_t o = 0;
        for (int axis = 0; axis < 3; axis++) {
            AxisBins &B = m->bins[axis];
            BinAxis &X = P.a[axis];
            const int nb = B.n_bins;
            B.h_gp_off.assign(h_offs.begin() + o, h_offs.begin() + o + nb + 1);
            B.h_dof_off.assign(h_offs.begin() + o + nb + 1, h_offs.begin() + o + 2 * (nb + 1));
            o += 2 * (nb + 1);
            B.n_tmpl = B.h_dof_off[nb];
            B.max_dof = 0;
            B.max_gp = 0;
            for (int b = 0; b < nb; b++) {
                B.max_dof = std::max(B.max_dof, B.h_dof_off[b + 1] - B.h_dof_off[b]);
                B.max_gp = std::max(B.max_gp, B.h_gp_off[b + 1] - B.h_gp_off[b]);
            }
            if (B.max_dof > kMaxBinItems || B.max_gp > kMaxBinItems)
                return set_error(FEM3_E_ARG, "a transverse bin holds more than 4096 dofs or "
                                             "Gauss points; lower fem3_options.bin_scale");
            max_gp = std::max(max_gp, B.max_gp);
            max_dof = std::max(max_dof, B.max_dof);
            FEM3_TRY(dev_alloc_t(m, &X.gkeys, n_gp));
            FEM3_TRY(dev_alloc_t(m, &X.dkeys, std::max<int64_t>(1, B.n_tmpl)));
            FEM3_TRY(dev_alloc_t(m, &X.dq, std::max<int64_t>(1, n_dof)));
            B.dof_key = X.dkeys;
            B.dof_q = X.dq;
            FEM3_TRY(dev_alloc_t(m, &B.gp_idx, n_gp));
            FEM3_TRY(dev_alloc_t(m, &B.slot_bin, n_gp));
            FEM3_TRY(dev_alloc_t(m, &B.dof_idx, std::max<int64_t>(1, B.n_tmpl)));
            FEM3_TRY(dev_alloc_t(m, &B.row_bin, std::max<int64_t>(1, B.n_tmpl)));
            FEM3_TRY(dev_alloc_t(m, &B.w_slot, n_gp));
            FEM3_TRY(dev_alloc_t(m, &B.slot_of_gp, n_gp));
            X.gp_idx = B.gp_idx;
            X.slot_bin = B.slot_bin;
            X.dof_idx = B.dof_idx;
            X.row_bin = B.row_bin;
            X.w_slot = B.w_slot;
            X.slot_of_gp = B.slot_of_gp;
        }
    }
    k_bin_fill3<<<dim3(gx, 3), kThreads, 0, s>>>(P, m->gp, n_gp, m->node_box, m->dof_node, n_dof);
    note_launch(m);
    {
        auto pow2 = [](int v) { int p = 1; while (p < v) p <<= 1; return p; };
        const size_t sh = sizeof(unsigned long long) * pow2(std::max(max_gp, max_dof));
        k_bin_sort3<<<dim3(nb_max, 3, 2), 256, sh, s>>>(P);
        note_launch(m);
    }
    k_bin_slots3<<<dim3(grid_for(n_gp), 3), kThreads, 0, s>>>(P, m->gw, n_gp);
    note_launch(m);

    for (int axis = 0; axis < 3; axis++) {
        AxisBins &B = m->bins[axis];
        const int nb = B.n_bins;
        // table layout: block of bin b is [D_b][ld_b], ld_b = Gauss points rounded up to 8
        B.h_tab_off.resize(nb);
        B.h_tab_ld.resize(nb);
        int64_t acc = 0;
        std::vector<int4> &work = B.h_work;
        work.clear();
        for (int b = 0; b < nb; b++) {
            int D = B.h_dof_off[b + 1] - B.h_dof_off[b];
            int Gc = B.h_gp_off[b + 1] - B.h_gp_off[b];
            int ld = (Gc + 7) & ~7;
            B.h_tab_off[b] = acc;
            B.h_tab_ld[b] = ld;
            acc += (int64_t)D * ld;
            if (D == 0 || Gc == 0) continue;
            int nt = (D + 63) / 64;
            for (int t1 = 0; t1 < nt; t1++)
                for (int t2 = t1; t2 < nt; t2++) work.push_back(make_int4(b, t1, t2, 0));
        }
        B.tab_elems = acc;
        B.n_work = (int)work.size();
        FEM3_TRY(dev_alloc_t(m, &B.tab_off, nb));
        FEM3_TRY(dev_alloc_t(m, &B.tab_ld, nb));
        FEM3_TRY(dev_alloc_t(m, &B.work, std::max(1, B.n_work)));
        FEM3_CUDA(cudaMemcpyAsync(B.tab_off, B.h_tab_off.data(), sizeof(int64_t) * nb,
                                  cudaMemcpyHostToDevice, s));
        FEM3_CUDA(cudaMemcpyAsync(B.tab_ld, B.h_tab_ld.data(), sizeof(int32_t) * nb,
                                  cudaMemcpyHostToDevice, s));
        if (B.n_work)
            FEM3_CUDA(cudaMemcpyAsync(B.work, work.data(), sizeof(int4) * B.n_work,
                                      cudaMemcpyHostToDevice, s));
        FEM3_TRY(dev_alloc_t(m, &m->tabL[axis], std::max<int64_t>(1, acc)));
        FEM3_TRY(dev_alloc_t(m, &m->tabR[axis], std::max<int64_t>(1, acc)));
    }
    FEM3_CUDA(cudaGetLastError());
    return FEM3_OK;
}

}  // namespace fem3
