// Allocation-free computation of the DFC correction factors lambda_k (Eq. 17)
// for one marker set, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need lambda_k:
// code running while a CUDA stream is being captured into a graph, host code
// inside a framework that owns every device allocation (and forbids others),
// or real-time loops where an allocation could block.  This entry point takes
// the caller's device input and output buffers and keeps its only scratch --
// W_total on the markers' bounding box -- in the file-scope array below.  It
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call rewrites every scratch node it reads, and clears the
// status word it reports through.  Calls that overlap on the GPU (different
// streams, or host threads racing) race on the array and must be serialised by
// the caller.
#include <cmath>
#include <mutex>

#include "iblbm.h"
#include "iblbm_dev.cuh"

namespace {

using namespace iblbm;

// W_total per node of the markers' bounding box: at most kNoAllocMaxBox nodes
// (2 MiB of FP64), i.e. a box of 512 x 512 nodes.
constexpr int kNoAllocMaxBox = 1 << 18;
static __device__ __align__(256) double g_noalloc_w[kNoAllocMaxBox];
// [0] status (0 ok, 1 box too large, 2 marker footprint outside the lattice),
// [1..4] box x0, y0, width, height.
static __device__ __align__(256) int g_noalloc_status[8];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_w_ptr[kMaxDevices] = {nullptr};
int* g_status_ptr[kMaxDevices] = {nullptr};

__device__ double phi_d(int kernel, double r) { return phi<double>(kernel, r); }

__device__ int stencil_origin(int kernel, double X) { return (int)floor(X) - (kernel == K_HAT ? 0 : 1); }

// One CTA: bounding box of all stencils, then W_total(x) = sum_k D(x - X_k)
// in ascending k at every box node, then W_sum(k) and lambda_k.
__global__ void __launch_bounds__(kThreads) noalloc_lambda_kernel(const double* __restrict__ xy, int n, double ds,
                                                                  int kernel, int nx, int ny, double* __restrict__ lam,
                                                                  double* w, int* status) {
    __shared__ int sh[4][kThreads];
    const int tid = threadIdx.x, S = kernel == K_HAT ? 2 : 4;
    int mnx = 1 << 30, mny = 1 << 30, mxx = -(1 << 30), mxy = -(1 << 30), bad = 0;
    for (int k = tid; k < n; k += kThreads) {
        const double X = xy[2 * k], Y = xy[2 * k + 1];
        const int i0 = stencil_origin(kernel, X), j0 = stencil_origin(kernel, Y);
        if (!(X == X) || !(Y == Y) || i0 < 0 || j0 < 0 || i0 + S > nx || j0 + S > ny) bad = 1;
        mnx = min(mnx, i0); mny = min(mny, j0); mxx = max(mxx, i0); mxy = max(mxy, j0);
    }
    __shared__ int shbad[kThreads];
    sh[0][tid] = mnx;
    sh[1][tid] = mny;
    sh[2][tid] = -mxx;   // maxima reduced as minima of the negatives
    sh[3][tid] = -mxy;
    shbad[tid] = bad;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            for (int q = 0; q < 4; ++q) sh[q][tid] = min(sh[q][tid], sh[q][tid + s]);
            shbad[tid] = max(shbad[tid], shbad[tid + s]);
        }
        __syncthreads();
    }
    const int bx0 = sh[0][0], by0 = sh[1][0], bw = -sh[2][0] + S - bx0, bh = -sh[3][0] + S - by0;
    if (shbad[0] || (long long)bw * bh > kNoAllocMaxBox) {
        if (tid == 0) status[0] = shbad[0] ? 2 : 1;
        return;
    }
    const int area = bw * bh;
    for (int q = tid; q < area; q += kThreads) {
        const int x = bx0 + q % bw, y = by0 + q / bw;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            const double dx = (double)x - xy[2 * k], dy = (double)y - xy[2 * k + 1];
            if (fabs(dx) >= S / 2 + 0.5 || fabs(dy) >= S / 2 + 0.5) continue;   // outside the stencil
            const int i0 = stencil_origin(kernel, xy[2 * k]), j0 = stencil_origin(kernel, xy[2 * k + 1]);
            if (x < i0 || x >= i0 + S || y < j0 || y >= j0 + S) continue;
            acc += phi_d(kernel, dx) * phi_d(kernel, dy);
        }
        w[q] = acc;
    }
    __syncthreads();
    for (int k = tid; k < n; k += kThreads) {
        const double X = xy[2 * k], Y = xy[2 * k + 1];
        const int i0 = stencil_origin(kernel, X), j0 = stencil_origin(kernel, Y);
        double ws = 0.0;
        for (int b = 0; b < S; ++b)
            for (int a = 0; a < S; ++a) {
                const double D = phi_d(kernel, (double)(i0 + a) - X) * phi_d(kernel, (double)(j0 + b) - Y);
                ws += w[(j0 + b - by0) * bw + (i0 + a - bx0)] * D;
            }
        lam[k] = 1.0 / (2.0 * 1.0 * ds * ws);
    }
    if (tid == 0) {
        status[1] = bx0; status[2] = by0; status[3] = bw; status[4] = bh;
    }
}

__global__ void noalloc_clear_status(int* status) {
    if (threadIdx.x < 8) status[threadIdx.x] = 0;
}

// Device addresses of the file-scope arrays, looked up once per device with
// that device current (host code cannot use the symbols' names as addresses).
int setup(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_w_ptr[dev] && g_status_ptr[dev]) return IBLBM_OK;
    void* w = nullptr;
    void* st = nullptr;
    if (cudaGetSymbolAddress(&w, g_noalloc_w) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    if (cudaGetSymbolAddress(&st, g_noalloc_status) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    g_w_ptr[dev] = static_cast<double*>(w);
    g_status_ptr[dev] = static_cast<int*>(st);
    return IBLBM_OK;
}

}  // namespace

extern "C" int iblbm_dfc_lambda_noalloc(const double* xy, int n, double ds, int kernel, int nx, int ny,
                                        double* lambda, void* stream) {
    if (!xy || !lambda || n <= 0 || !(ds > 0.0) || (kernel != K_HAT && kernel != K_P4) || nx < 1 || ny < 1)
        return IBLBM_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    int rc = setup(dev);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    IBLBM_LAUNCH(noalloc_clear_status, 1, 32, st, g_status_ptr[dev]);
    IBLBM_LAUNCH(noalloc_lambda_kernel, 1, kThreads, st, xy, n, ds, kernel, nx, ny, lambda, g_w_ptr[dev],
                 g_status_ptr[dev]);
    if (cudaGetLastError() != cudaSuccess) return IBLBM_ERR_CUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, g_status_ptr[dev], sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    if (status == 1) return IBLBM_ERR_CAPACITY;
    if (status == 2) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
    return IBLBM_OK;
}
