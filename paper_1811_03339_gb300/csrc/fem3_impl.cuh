// Internal declarations shared by the translation units of libfem3 (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fem3.h"

namespace fem3 {

// ---------------------------------------------------------------------------------
// error reporting (thread-local text, status codes from fem3.h)
// ---------------------------------------------------------------------------------
int set_error(int code, const std::string &msg);
int cuda_error(cudaError_t e, const char *where);

#define FEM3_CUDA(call)                                                        \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::fem3::cuda_error(e_, #call);           \
    } while (0)

#define FEM3_TRY(call)                                                         \
    do {                                                                       \
        int s_ = (call);                                                       \
        if (s_ != FEM3_OK) return s_;                                          \
    } while (0)

// Error words written by kernels (device int32 array in the handle).
enum ErrWord {
    ERR_WALK = 0,      // number of walks that exceeded the step cap or found no exit
    ERR_TEMPLATE = 1,  // number of table updates whose dof was not in the bin's template
    ERR_NOT_SPD = 2,   // 1 + first column with a non-positive pivot (0: none)
    ERR_MESH = 3,      // number of degenerate tets
    ERR_FACE = 4,      // non-manifold faces or hash overflow
    ERR_SOLVE = 5,     // a triangular-solve wait gave up (bounded spin)
    ERR_TC = 6,        // a tensor-core contraction pipeline wait gave up
    ERR_CHOL = 7,      // a tile-factorisation wait gave up (bounded spin)
    ERR_COUNT = 8
};

// Walk tolerances (the paper's exact zero tests, made relative).  The CPU oracle uses
// the same constants; nothing is shared between the two code bases but the numbers.
constexpr double kEpsLambda = 1e-12;  // zero test of a volume coordinate
constexpr double kEpsRRel = 1e-12;    // segment-length / tie tolerance, times the mesh span
constexpr double kEpsDRel = 1e-12;    // |gradient| below this fraction of the largest: parallel

constexpr int kMaxBinItems = 4096;    // max dofs or Gauss points in one transverse bin
constexpr int kSegCounterSlot = 120;  // norms[120]: segment counter (norms[0..63] reductions)
                                      // norms[121]: contraction work counter

// Transverse bins of one axis: the plane of the two other coordinates is cut into an
// nb0 x nb1 grid; a Gauss point belongs to the bin of its transverse position, a dof
// to every bin its element patch's transverse bounding box meets (template set).
struct AxisBins {
    int c0 = 0, c1 = 0;          // transverse coordinates (c0 < c1)
    int nb0 = 0, nb1 = 0, n_bins = 0;
    double org0 = 0, org1 = 0, width = 0;
    int32_t *gp_off = nullptr;   // [n_bins+1]   bin -> slots
    int32_t *gp_idx = nullptr;   // [n_gp]       slot -> Gauss point (sorted along the axis)
    int32_t *slot_bin = nullptr; // [n_gp]       slot -> bin
    int32_t *slot_of_gp = nullptr; // [n_gp]     Gauss point -> slot
    double *w_slot = nullptr;    // [n_gp]       Gauss weight of each slot
    int32_t *dof_off = nullptr;  // [n_bins+1]
    int32_t *dof_idx = nullptr;  // [n_tmpl]     dof ids per bin, sorted by dof_key
    // [n_tmpl] row keys: (lower end of the dof's element patch along the axis, quantised to
    // 30 bits) << 32 | dof id, ascending within a bin; [n_dof] that quantised position
    unsigned long long *dof_key = nullptr;
    uint32_t *dof_q = nullptr;
    // [n_tmpl] Gauss-point ranges [first, end) of the nonzeros of each row of L and of R
    // (x, y: L; z, w: R), written with the apply operands
    int4 *ap_rng = nullptr;
    // the nonzeros of L and W R (t = 0: L, 1: W R) as lists, written with the apply operands:
    // row-major, a template row's list in the place of its dense table row (Gauss-point index
    // in the bin, value), and Gauss-point major in chunks of 32 points within the bin's block
    // (row index in the bin, value; layout at k_gp_lists); list lengths per template row and
    // per Gauss-point slot
    uint16_t *rl_g[2] = {nullptr, nullptr};
    float2 *rl_v[2] = {nullptr, nullptr};
    int32_t *rl_n[2] = {nullptr, nullptr};
    uint16_t *gl_r[2] = {nullptr, nullptr};
    float2 *gl_v[2] = {nullptr, nullptr};
    int32_t *gl_n[2] = {nullptr, nullptr};
    int64_t *tab_off = nullptr;  // [n_bins]     element offset of the bin's table block
    int32_t *tab_ld = nullptr;   // [n_bins]     leading dimension (padded Gauss-point count)
    int64_t n_tmpl = 0, tab_elems = 0;
    int max_dof = 0, max_gp = 0;
    int4 *work = nullptr;        // contraction work items (bin, t1, t2, 0)
    int n_work = 0;
    int4 *form_work = nullptr;   // general-form work items: every tile pair (bin, t1, t2, 0)
    int n_form_work = 0;
    // tensor-core contraction operands: TF32 or BF16 hi/lo of L and of W R, [n_tmpl][Kp]
    // (Kp = tc_maxG rounded to one 128-byte row of the operand type)
    void *tc_op[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t *row_bin = nullptr;  // [n_tmpl] template row -> bin
    int tc_maxG = 0;             // largest Gauss-point count of a bin
    int4 *tc_work[2] = {nullptr, nullptr};   // (bin, m-tile, n-tile, 0) per tile width
    // operator-apply operand W R as hi + lo FP32 pairs in the table layout (L is the table)
    float2 *ap_R = nullptr;
    int tc_n_work[2] = {0, 0};
    std::vector<int32_t> h_gp_off, h_dof_off;
    std::vector<int4> h_work, h_tc_work[2];   // host copies of the work lists
    std::vector<int64_t> h_tab_off;
    std::vector<int32_t> h_tab_ld;
};

struct Mesh {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t n_nodes = 0, n_tets = 0, n_gp = 0, n_dof = 0;
    double span = 0, h_est = 0, bin_scale = 1.0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int max_steps = 0;
    bool profile = false;

    // geometry (device)
    double *verts = nullptr;   // [n_nodes][3]
    int32_t *tets = nullptr;   // [n_tets][4]
    double *M = nullptr;       // [n_tets][16] rows (c_k, dlam_k/dx, dlam_k/dy, dlam_k/dz)
    double *inv = nullptr;     // [n_tets][3][4] 1/dlam_k/dx_axis, 0 if parallel
    float4 *recf = nullptr;    // [n_tets][3][8] FP32 records of the walk's exit filter
    double *vol = nullptr;     // [n_tets]
    int32_t *nbr = nullptr;    // [n_tets][4]
    int32_t *dof = nullptr;    // [n_nodes]
    int32_t *dof_node = nullptr;  // [n_dof]
    int32_t *vt_off = nullptr;    // [n_nodes+1]
    int32_t *vt_tet = nullptr;    // [4 n_tets]
    double *gp = nullptr;      // [n_gp][3]
    double *gw = nullptr;      // [n_gp]
    double *node_box = nullptr;   // [n_nodes][6] patch bounding box (lo xyz, hi xyz)
    int32_t *err = nullptr;    // [ERR_COUNT]

    AxisBins bins[3];
    // derivative tables L, R as unevaluated hi + lo FP32 pairs (value = x + y)
    float2 *tabL[3] = {nullptr, nullptr, nullptr};
    float2 *tabR[3] = {nullptr, nullptr, nullptr};
    float2 *pow_cell = nullptr;   // [3][256][8] tables of the table-driven power (hi + lo pairs)
    float2 *pow_exp = nullptr;    // [3][128]

    // assembled operator
    int precision = -1;        // of the last assemble, -1: none
    double alpha[3] = {0, 0, 0}, K[3] = {0, 0, 0};
    double s[3] = {0, 0, 0};   // Riesz constants s_i = 1/(2 cos(pi alpha_i/2))
    double sK[3] = {0, 0, 0};  // s_i K_i
    double *A64 = nullptr;     // [n_dof][n_dof]
    float *A32 = nullptr;      // [n_dof][n_dof]
    bool factored = false;
    bool tc_ready = false;
    int tc_tile_opt = 0;       // tensor-core tile width asked for: 0 tuned, 128 or 256
    int tc_tile_used = 0;      // width of the last tensor-core contraction
    bool tc_tuned = false;     // the last contraction ran the tuner
    bool ap_ready = false;     // ap_R holds W R of the current tables
    bool integer_order = false;   // the matrix came from fem3_assemble_integer (no tables)
    double *form_wc = nullptr;    // general form: w c per Gauss point, and per slot of one axis
    double *A_ns = nullptr;       // divergence-form (non-symmetric) matrix, FP64 [n_dof][n_dof]
    bool nonsym = false;          // the current operator is A_ns (GMRES solve)
    int part = 0, nparts = 1;     // assembly restricted to part `part` of every axis's bins

    // workspaces
    double *vec64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    float *vec32[2] = {nullptr, nullptr};
    int32_t *flags = nullptr;  // triangular-solve flags: [2 nblk + 2]
    void *solve_ws = nullptr;  // triangular-solve z blocks: nblk x 64 x 24 doubles
    void *solve_G = nullptr;   // triangular-solve chain operators: nblk x 2 x 3 x 64 x 64 doubles
    int32_t *chol_flags = nullptr;  // tile-factorisation flags, then ticket and abort words
    void *dinv = nullptr;      // inverses of the 64 x 64 diagonal blocks of the factor
    float *chol_w = nullptr;   // tensor-core factorisation: TF32 hi / lo operand rows, panel inverse
    int64_t chol_w_rows = 0;
    int chol_tc_opt = 0;       // 0: by size, 1: always, -1: never (tensor-core factorisation)
    bool chol_tc_used = false; // the last factorisation ran on the tensor cores
    int flag_epoch = 0;        // value that marks "ready" in the current solve
    double *norms = nullptr;   // device scratch for reductions
    double *h_norms = nullptr; // pinned host mirror

    // counters
    int64_t launches = 0;      // kernels this handle has launched
    int64_t segments = 0;
    double contract_flops = 0;

    // profiling
    cudaEvent_t ev[16];
    bool ev_made = false;
    float stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // per kernel class (KernelClass): event pairs around each launch, summed when collected
    std::vector<cudaEvent_t> kc_ev;
    std::vector<int> kc_cls;
    size_t kc_used = 0;
    float kc_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int32_t kc_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};

    std::vector<void *> allocs;   // stream-ordered allocations, freed with the mesh
    char *arena = nullptr;        // current sub-allocation chunk (one of allocs)
    size_t arena_size = 0, arena_used = 0;
};

inline void note_launch(Mesh *m) { m->launches++; }

// bins [b0, b1) of the current part of an axis: contiguous ranges of equal bin count
inline void part_bins(const Mesh *m, int axis, int &b0, int &b1) {
    const int64_t nb = m->bins[axis].n_bins;
    b0 = (int)(nb * m->part / m->nparts);
    b1 = (int)(nb * (m->part + 1) / m->nparts);
}

// device memory owned by a mesh (stream-ordered pool allocations)
int dev_alloc(Mesh *m, void **p, size_t bytes);
template <class T>
int dev_alloc_t(Mesh *m, T **p, size_t n) {
    return dev_alloc(m, reinterpret_cast<void **>(p), n * sizeof(T) > 0 ? n * sizeof(T) : 16);
}
void dev_free_all(Mesh *m);

// true if p is device or managed memory
bool is_device_ptr(const void *p);

// profiling helpers
void stage_begin(Mesh *m, int stage);
void stage_end(Mesh *m, int stage);
void stage_collect(Mesh *m);

// Kernel classes timed one launch at a time when the mesh profiles (fem3_kernel_ms):
// CUDA events on the launch stream around every launch of the class.
enum KernelClass {
    KC_WALK = 0,      // k_walk_tables: walk + derivative tables, three axes in one launch
    KC_SPLIT = 1,     // k_split_ops: operand split of the tables
    KC_CONTRACT = 2,  // contraction GEMMs (tensor-core or CUDA-core)
    KC_FACTOR = 3,    // Cholesky factorisation
    KC_CHAIN = 4,     // triangular-solve chains
    KC_APPLY = 5,     // operator apply of the refinement residual
    KC_COUNT = 6
};
void kc_begin(Mesh *m, int cls);
void kc_end(Mesh *m, int cls);
void kc_reset(Mesh *m);

// exclusive scan of int32 counts into offsets [n+1]; returns total via device offsets[n]
int scan_i32(const int32_t *in, int32_t *out, int64_t n, cudaStream_t s, Mesh *m);

// scratch of the batched walk (descriptor arrays; freed by the batch)
// row-major lists of a table pair (L, W R) as k_split_ops writes them (null: not written)
struct RowLists {
    uint16_t *g0, *g1;   // Gauss-point index in the bin
    float2 *v0, *v1;     // L, W R values (hi + lo)
    int32_t *n0, *n1;    // [n_tmpl] lengths
};

struct BatchWalkScratch {
    void *d_desc = nullptr, *h_desc = nullptr;
};

// one mesh of a batched triangular solve (device-resident descriptor)
struct BatchTrsmDesc {
    const void *L;      // factor, row-major n x n (float or double)
    const void *dinv;   // inverses of the 64 x 64 diagonal blocks
    void *y;            // right-hand sides / solutions, column-major [n][nrhs]
    int64_t n;
    int nblk;
    int active;         // 0: skip this mesh
};

// translation-unit entry points
int mesh_build(Mesh *m, const double *verts_d, const int32_t *tets_d);
int bins_build(Mesh *m);
int walk_tables(Mesh *m, const double alpha[3]);
int walk_tables_batch(Mesh *const *ms, int n, const double *alpha, cudaStream_t s,
                      BatchWalkScratch *bs);
int walk_paths(Mesh *m, int axis, int dir, const int64_t *gps, int64_t n, int cap,
               int32_t *tet_out, double *r0, double *r1, int32_t *nseg);
int table_rows(Mesh *m, int axis, int dir, const int64_t *gps, int64_t n, double *rows);
int contract(Mesh *m, int precision);
int contract_tc(Mesh *m, bool bf16);   // TF32 x 3 (bf16 = false) or BF16 x 3
// algorithmic flops of the element sum and nonzeros of the tables (synchronises)
int contract_work(Mesh *m, double *flops, int64_t *nnz);
// general form (c D^a u, D^^b v) of one axis
int walk_tables_form(Mesh *m, int axis, double order_left, double order_right);
int weight_coef(Mesh *m, const double *c_gp, double *wc_gp);   // wc = w c per Gauss point
int contract_form(Mesh *m, int axis, bool test_right, const double *wc_gp, int precision);
int contract_tc_form(Mesh *m, int axis, bool test_right, double *wc_gp, bool bf16);
int load_vector(Mesh *m, const double *f_d, int nrhs, double *b_d);
int load_vector_T(Mesh *m, const double *lam_d, double *out_d);
int factor(Mesh *m);
int chol_tc(Mesh *m, float *A, int64_t n);
int assemble_integer(Mesh *m, const double K[3]);       // P1 stiffness, alpha_i = 2
int axis_forms_integer(Mesh *m, const double *u, const double *lam, double out[3]);
int apply_integer(Mesh *m, const double *x, double *y); // y = A x, element by element
int assemble_divergence(Mesh *m, const double beta[3], const double *p_d, const double *q_d,
                        int precision);
int factor_nonsym(Mesh *m);   // FP64 Cholesky of -(A + A^T)/2: the GMRES preconditioner
int gmres_solve(Mesh *m, const double *b, double *x, double tol, int max_iter, int *iters,
                double *resid);   // blocked FP32 Cholesky, tcgen05 trailing updates
int solve_direct(Mesh *m, const double *b_d, int nrhs, double *u_d);
int solve_refined(Mesh *m, const double *b_d, int nrhs, double tol, int max_iter, double *u_d,
                  int *iters, double *resid);
int apply_A64(Mesh *m, const double *u_d, double *Au_d);
int axis_forms(Mesh *m, const double *u_d, const double *lam_d, double out[3]);
int read_errors(Mesh *m, int32_t *h_err);
int trsm_batch(const BatchTrsmDesc *d_desc, int n_mesh, int max_nblk, int nrhs, bool fp64,
               cudaStream_t s);
int apply_multi(Mesh *m, const double *u_d, int nv, double *Au_d, bool df = true);
int f32_to_f64(const float *a, double *b, int64_t n, cudaStream_t s);
int sym_from_lower(double *A, int64_t n, cudaStream_t s);
int sub_vec(const double *a, const double *b, double *c, int64_t n, cudaStream_t s);
// rel = ||b - Au|| / ||b|| (synchronises)
int residual_norm(Mesh *m, const double *b, const double *Au, double *rel);

int ap_alloc(Mesh *m, int axis);   // operator-apply operand buffers of one axis
int ap_prepare(Mesh *m);           // split the current tables into the apply operands
// The operator apply runs from the lists of the tables' nonzeros when a bin's u rows and its
// Gauss points' sums of 17 vectors fit the list kernel's shared memory and its rows its
// threads' items (kListItems per thread, two vector groups); otherwise from the dense table
// blocks (with the W R operand in the table layout)
constexpr size_t kListSmemMax = 112 * 1024;   // two CTAs per SM at least
constexpr int kListItems = 2;                  // phase-2 items (row, vector group) per thread
inline size_t apply_lists_smem(int nr, int max_dof, int max_gp) {
    return 8 * (size_t)nr * ((size_t)max_dof + (size_t)max_gp);
}
inline bool apply_lists_fit(const Mesh *m) {
    int md = 0, mg = 0;
    for (int a = 0; a < 3; a++) {
        md = std::max(md, m->bins[a].max_dof);
        mg = std::max(mg, m->bins[a].max_gp);
    }
    return apply_lists_smem(17, md, mg) <= kListSmemMax && 2 * md <= 256 * kListItems;
}
RowLists row_lists(AxisBins &B);   // the axis's row-major list arrays
void launch_gp_lists(Mesh *m, int axis);   // Gauss-point-major lists of L and W R

// ---------------------------------------------------------------------------------
// FP64 values in FP32 arithmetic.  GB300 runs FP64 arithmetic and f64 <-> f32
// conversions at 1/64 of the FP32 rate, so the operator apply keeps FP64 only as the
// storage format: values are split into unevaluated sums hi + lo of two FP32 numbers by
// integer operations and products are accumulated in that form.
// ---------------------------------------------------------------------------------
// hi: leading 24 bits of the significand (truncated); lo: the next 29 bits rounded to 24.
// |x - hi - lo| <= 2^-48 |x| for 2^-74 <= |x| < 2^128; below 2^-74 lo = 0, below 2^-126
// both are (signed) zero.
__device__ __forceinline__ void f64_split(double x, float &hi, float &lo) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
    const uint32_t ef = static_cast<uint32_t>(b >> 52) & 0x7FFu;
    const float zero = __uint_as_float(sign);
    if (ef < 897u) {
        hi = zero;
        lo = zero;
        return;
    }
    hi = __uint_as_float(sign | ((ef - 896u) << 23) | (static_cast<uint32_t>(b >> 29) & 0x7FFFFFu));
    const uint32_t rest = static_cast<uint32_t>(b) & 0x1FFFFFFFu;
    if (ef < 949u || rest == 0) {
        lo = zero;
        return;
    }
    // rest = rh 2^23 + rl with both parts exact in FP32 (2^23 + m has the bits of m)
    const float rh = __uint_as_float(0x4B000000u | (rest >> 23)) - 8388608.0f;
    const float rl = __uint_as_float(0x4B000000u | (rest & 0x7FFFFFu)) - 8388608.0f;
    const float mag = fmaf(rh, 8388608.0f, rl) * __uint_as_float((ef - 948u) << 23);
    lo = __uint_as_float(__float_as_uint(mag) | sign);
}

// (sh, sl) += (ah + al)(bh + bl): ah bh exactly as p + e (FMA), the cross terms in FP32
// (their rounding is 2^-24 of a 2^-24-sized term), al bl dropped, p added by TwoSum.
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float &sh, float &sl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    const float x = fmaf(ah, bl, al * bh);
    const float t = sh + p;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (p - z);
    sh = t;
    sl += err + (e + x);
}

// (sh, sl) += (bh, bl)
__device__ __forceinline__ void df_add(float bh, float bl, float &sh, float &sl) {
    const float t = sh + bh;
    const float z = t - sh;
    const float err = (sh - (t - z)) + (bh - z);
    sh = t;
    sl += err + bl;
}

// (rh, rl) = (ah + al)(bh + bl), normalised (|rl| <= ulp(rh) / 2)
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &rh, float &rl) {
    const float p = ah * bh;
    const float e = fmaf(ah, bh, -p);
    const float x = fmaf(ah, bl, al * bh) + e;
    rh = p + x;
    rl = x - (rh - p);
}

// (rh, rl) = (ah + al) + (bh + bl), normalised
__device__ __forceinline__ void df_add2(float ah, float al, float bh, float bl, float &rh, float &rl) {
    const float t = ah + bh;
    const float z = t - ah;
    const float x = ((ah - (t - z)) + (bh - z)) + (al + bl);
    rh = t + x;
    rl = x - (rh - t);
}

// exact FP32 value of an integer |v| <= 2^22 without a conversion instruction:
// 1.5 * 2^23 + v has the bits of the magic constant plus v
__device__ __forceinline__ float small_int_f32(int v) {
    return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

}  // namespace fem3
