// fem3_spd_solve_static: a dense SPD solve that allocates no device memory.
//
// Some callers cannot allocate device memory at the point where they need a solve:
// latency-critical loops that must never enter the allocator, and host applications or
// plugin hosts that own every device allocation themselves and hand the library only the
// buffers of the problem.  This entry point serves them: its working memory (the
// Cholesky factor, the inverse of the current 64 x 64 diagonal block and an error word)
// is one file-scope static device array, so the caller passes only the matrix, the
// right-hand side and the output.  Each call ends by reading the error word back and
// synchronising its stream.
//
// The factorisation is its own multi-launch blocked right-looking Cholesky (64-wide
// blocks: diagonal factor and inverse, panel product, trailing update of the lower
// triangle, one launch each per block column) followed by blocked forward and backward
// substitution.  It shares no kernel with fem3_solve, whose FP64 form serves only as the
// reference in the test of this entry point.
#include <math.h>

#include <mutex>

#include "fem3_impl.cuh"

namespace fem3 {

namespace {

constexpr int kNaMaxN = 512;   // largest system this entry point accepts
constexpr int NBS = 64;

// factor [kNaMaxN^2] | diagonal-block inverse [64*64] | error word (as 8 doubles)
constexpr size_t kNaFactor = (size_t)kNaMaxN * kNaMaxN;
constexpr size_t kNaElems = kNaFactor + NBS * NBS + 8;
static __device__ __align__(256) double g_na_scratch[kNaElems];

std::mutex g_na_mutex;
void *g_na_ptr[256];   // per device: device address of g_na_scratch (host-side table)

// F = A (row-major n x n), x = b
__global__ void k_na_copy(const double *__restrict__ A, const double *__restrict__ b, int n,
                          double *F, double *x) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < (int64_t)n * n) F[i] = A[i];
    if (i < n) x[i] = b[i];
}

__global__ void __launch_bounds__(256) k_na_potrf_inv(double *F, int n, int k0, double *Linv,
                                                      int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double(*a)[NBS + 1] = reinterpret_cast<double(*)[NBS + 1]>(smem_raw);
    double(*li)[NBS + 1] = a + NBS;
    const int nb = min(NBS, n - k0);
    for (int e = threadIdx.x; e < NBS * NBS; e += blockDim.x) {
        int i = e / NBS, j = e % NBS;
        a[i][j] = (i < nb && j < nb) ? F[(int64_t)(k0 + i) * n + k0 + j] : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int j = 0; j < nb; j++) {
        if (threadIdx.x == 0) {
            double d = a[j][j];
            if (!(d > 0.0)) {
                atomicCAS(err, 0, k0 + j + 1);
                d = 1.0;
            }
            a[j][j] = sqrt(d);
        }
        __syncthreads();
        double djj = a[j][j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= djj;
        __syncthreads();
        const int m = nb - j - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = j + 1 + e / m, c = j + 1 + e % m;
            if (c <= i) a[i][c] -= a[i][j] * a[c][j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        int i = e / nb, j = e % nb;
        F[(int64_t)(k0 + i) * n + k0 + j] = j <= i ? a[i][j] : 0.0;
    }
    if (threadIdx.x < NBS) {
        const int c = threadIdx.x;
        for (int r = 0; r < NBS; r++) li[r][c] = 0.0;
        li[c][c] = 1.0 / a[c][c];
        for (int r = c + 1; r < NBS; r++) {
            double s = 0.0;
            for (int k = c; k < r; k++) s += a[r][k] * li[k][c];
            li[r][c] = -s / a[r][r];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NBS * NBS; e += blockDim.x) Linv[e] = li[e / NBS][e % NBS];
}

__global__ void __launch_bounds__(256) k_na_trsm(double *F, int n, int k0, const double *Linv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double(*bt)[NBS + 1] = reinterpret_cast<double(*)[NBS + 1]>(smem_raw);
    double(*li)[NBS + 1] = bt + NBS;
    const int row0 = k0 + NBS + blockIdx.x * NBS;
    for (int e = threadIdx.x; e < NBS * NBS; e += blockDim.x) {
        int i = e / NBS, j = e % NBS;
        bt[i][j] = (row0 + i < n) ? F[(int64_t)(row0 + i) * n + k0 + j] : 0.0;
        li[i][j] = Linv[e];
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k = 0; k < NBS; k++)
        for (int p = 0; p < 4; p++)
            for (int q = 0; q < 4; q++) acc[p][q] = fma(bt[ty * 4 + p][k], li[tx * 4 + q][k], acc[p][q]);
    for (int p = 0; p < 4; p++) {
        int r = row0 + ty * 4 + p;
        if (r >= n) continue;
        for (int q = 0; q < 4; q++) F[(int64_t)r * n + k0 + tx * 4 + q] = acc[p][q];
    }
}

__global__ void __launch_bounds__(256) k_na_syrk(double *F, int n, int k0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double(*pi)[NBS + 1] = reinterpret_cast<double(*)[NBS + 1]>(smem_raw);
    double(*pj)[NBS + 1] = pi + NBS;
    int idx = blockIdx.x, ti = 0;
    while (idx > ti) { idx -= ti + 1; ti++; }
    const int tj = idx;
    const int i0 = k0 + NBS + ti * NBS, j0 = k0 + NBS + tj * NBS;
    for (int e = threadIdx.x; e < NBS * NBS; e += blockDim.x) {
        int r = e / NBS, c = e % NBS;
        pi[r][c] = (i0 + r < n) ? F[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
        pj[r][c] = (j0 + r < n) ? F[(int64_t)(j0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int c = 0; c < NBS; c++)
        for (int a = 0; a < 4; a++)
            for (int b = 0; b < 4; b++) acc[a][b] = fma(pi[ty * 4 + a][c], pj[tx * 4 + b][c], acc[a][b]);
    for (int a = 0; a < 4; a++) {
        int r = i0 + ty * 4 + a;
        if (r >= n) continue;
        for (int b = 0; b < 4; b++) {
            int c = j0 + tx * 4 + b;
            if (c < n && c <= r) F[(int64_t)r * n + c] -= acc[a][b];
        }
    }
}

// substitution on one 64-row block by one warp (backward = 1 uses the transpose)
__global__ void k_na_trsv_diag(const double *F, int n, int k0, double *y, int backward) {
    const int nb = min(NBS, n - k0), lane = threadIdx.x;
    double t0 = lane < nb ? y[k0 + lane] : 0.0, t1 = lane + 32 < nb ? y[k0 + lane + 32] : 0.0;
    if (!backward) {
        for (int c = 0; c < nb; c++) {
            double tc = c < 32 ? __shfl_sync(0xffffffffu, t0, c) : __shfl_sync(0xffffffffu, t1, c - 32);
            double v = tc / F[(int64_t)(k0 + c) * n + k0 + c];
            if (lane == (c & 31)) { if (c < 32) t0 = v; else t1 = v; }
            if (lane > c && lane < nb) t0 -= F[(int64_t)(k0 + lane) * n + k0 + c] * v;
            if (lane + 32 > c && lane + 32 < nb) t1 -= F[(int64_t)(k0 + lane + 32) * n + k0 + c] * v;
        }
    } else {
        for (int c = nb - 1; c >= 0; c--) {
            double tc = c < 32 ? __shfl_sync(0xffffffffu, t0, c) : __shfl_sync(0xffffffffu, t1, c - 32);
            double v = tc / F[(int64_t)(k0 + c) * n + k0 + c];
            if (lane == (c & 31)) { if (c < 32) t0 = v; else t1 = v; }
            if (lane < c) t0 -= F[(int64_t)(k0 + c) * n + k0 + lane] * v;
            if (lane + 32 < c) t1 -= F[(int64_t)(k0 + c) * n + k0 + lane + 32] * v;
        }
    }
    if (lane < nb) y[k0 + lane] = t0;
    if (lane + 32 < nb) y[k0 + lane + 32] = t1;
}

// forward: rows below the block; backward: rows above the block
__global__ void k_na_trsv_update(const double *F, int n, int k0, double *y, int backward) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nb = min(NBS, n - k0);
    double s = 0.0;
    if (!backward) {
        if (i < k0 + nb || i >= n) return;
        for (int c = 0; c < nb; c++) s += F[(int64_t)i * n + k0 + c] * y[k0 + c];
    } else {
        if (i >= k0) return;
        for (int c = 0; c < nb; c++) s += F[(int64_t)(k0 + c) * n + i] * y[k0 + c];
    }
    y[i] -= s;
}

// device address of the static scratch for the current device (set up once per device)
int na_scratch(double **out) {
    int dev = 0;
    FEM3_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(FEM3_E_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        const size_t sh = 2 * NBS * (NBS + 1) * sizeof(double);
        FEM3_CUDA(cudaFuncSetAttribute(k_na_potrf_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        FEM3_CUDA(cudaFuncSetAttribute(k_na_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        FEM3_CUDA(cudaFuncSetAttribute(k_na_syrk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
        g_na_ptr[dev] = p;
    }
    *out = static_cast<double *>(g_na_ptr[dev]);
    return FEM3_OK;
}

// true if p is device (or managed) memory that the current device can use directly
bool on_current_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

}  // namespace fem3

using namespace fem3;

extern "C" int fem3_spd_solve_static(const double *A, int64_t n, const double *b, double *x,
                                     void *stream) {
    if (!A || !b || !x) return set_error(FEM3_E_ARG, "null argument");
    if (n < 1 || n > kNaMaxN)
        return set_error(FEM3_E_ARG, "fem3_spd_solve_static accepts 1 <= n <= 512 (its static "
                                     "working memory holds one 512 x 512 factor)");
    // the kernels read A and b and write x directly: all three must be device memory of
    // the current device (a host or foreign-device pointer is rejected, never dereferenced)
    if (!on_current_device(A) || !on_current_device(b) || !on_current_device(x))
        return set_error(FEM3_E_ARG, "fem3_spd_solve_static: A, b and x must be device memory "
                                     "of the current device");
    double *scratch = nullptr;
    FEM3_TRY(na_scratch(&scratch));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double *F = scratch;
    double *Linv = scratch + kNaFactor;
    int *err = reinterpret_cast<int *>(scratch + kNaFactor + NBS * NBS);
    const int nn = (int)n;
    const size_t sh = 2 * NBS * (NBS + 1) * sizeof(double);
    // the error word must start at zero; the factor and inverse are fully rewritten
    FEM3_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_na_copy<<<(unsigned)((n * n + 255) / 256), 256, 0, s>>>(A, b, nn, F, x);
    for (int k0 = 0; k0 < nn; k0 += NBS) {
        k_na_potrf_inv<<<1, 256, sh, s>>>(F, nn, k0, Linv, err);
        const int rest = nn - k0 - NBS;
        if (rest > 0) {
            const int nblk = (rest + NBS - 1) / NBS;
            k_na_trsm<<<nblk, 256, sh, s>>>(F, nn, k0, Linv);
            k_na_syrk<<<nblk * (nblk + 1) / 2, 256, sh, s>>>(F, nn, k0);
        }
    }
    for (int k0 = 0; k0 < nn; k0 += NBS) {
        k_na_trsv_diag<<<1, 32, 0, s>>>(F, nn, k0, x, 0);
        if (k0 + NBS < nn) k_na_trsv_update<<<(nn + 255) / 256, 256, 0, s>>>(F, nn, k0, x, 0);
    }
    for (int k0 = ((nn - 1) / NBS) * NBS; k0 >= 0; k0 -= NBS) {
        k_na_trsv_diag<<<1, 32, 0, s>>>(F, nn, k0, x, 1);
        if (k0 > 0) k_na_trsv_update<<<(k0 + 255) / 256, 256, 0, s>>>(F, nn, k0, x, 1);
    }
    FEM3_CUDA(cudaGetLastError());
    int h_err = 0;
    FEM3_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEM3_CUDA(cudaStreamSynchronize(s));
    if (h_err)
        return set_error(FEM3_E_NOT_SPD,
                         "non-positive pivot in Cholesky at column " + std::to_string(h_err - 1));
    return FEM3_OK;
}
