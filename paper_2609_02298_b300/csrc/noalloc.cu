// Allocation-free computation of the DFC correction factors lambda_k (Eq. 17)
// for one marker set, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need lambda_k:
// host code inside a framework that owns every device allocation (and forbids
// others), solvers embedded in another application's time loop where an
// allocation would synchronise the device or could fail mid-run, or real-time
// loops where an allocation could block.  This entry point takes the caller's
// device input and output buffers and keeps its only scratch -- W_total on the
// markers' bounding box -- in the file-scope array below.  It allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library call.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call rewrites every scratch node it reads, and rewrites the
// status word it reports through before anything reads it.  Calls that overlap
// on the GPU (different streams, or host threads racing) race on the array and
// must be serialised by the caller.
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
constexpr int kTileW = 32, kTileH = kThreads / kTileW;   // box tile of one CTA pass (32 x 8 nodes)
constexpr int kWGrid = 148 * 4;                            // CTAs of the W_total pass (grid-stride over tiles)
std::mutex g_mu;
double* g_w_ptr[kMaxDevices] = {nullptr};
int* g_status_ptr[kMaxDevices] = {nullptr};

__device__ double phi_d(int kernel, double r) { return phi<double>(kernel, r); }

__device__ int stencil_origin(int kernel, double X) { return (int)floor(X) - (kernel == K_HAT ? 0 : 1); }

// Pass 1 (one CTA): bounding box of all stencils and the validity of every
// footprint; writes the status word and the box for the two passes after it.
__global__ void __launch_bounds__(kThreads) noalloc_box_kernel(const double* __restrict__ xy, int n, int kernel,
                                                               int nx, int ny, int* status) {
    __shared__ int sh[5][kThreads];
    const int tid = threadIdx.x, S = kernel == K_HAT ? 2 : 4;
    int mnx = 1 << 30, mny = 1 << 30, mxx = -(1 << 30), mxy = -(1 << 30), bad = 0;
    for (int k = tid; k < n; k += kThreads) {
        const double X = xy[2 * k], Y = xy[2 * k + 1];
        if (!(X == X) || !(Y == Y) || fabs(X) > 1e9 || fabs(Y) > 1e9) {
            bad = 1;
            continue;
        }
        const int i0 = stencil_origin(kernel, X), j0 = stencil_origin(kernel, Y);
        if (i0 < 0 || j0 < 0 || i0 + S > nx || j0 + S > ny) bad = 1;
        mnx = min(mnx, i0); mny = min(mny, j0); mxx = max(mxx, i0); mxy = max(mxy, j0);
    }
    sh[0][tid] = mnx;
    sh[1][tid] = mny;
    sh[2][tid] = -mxx;   // maxima reduced as minima of the negatives
    sh[3][tid] = -mxy;
    sh[4][tid] = -bad;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (tid < s)
            for (int q = 0; q < 5; ++q) sh[q][tid] = min(sh[q][tid], sh[q][tid + s]);
        __syncthreads();
    }
    if (tid == 0) {
        const int bx0 = sh[0][0], by0 = sh[1][0];
        const long long bw = (long long)(-sh[2][0]) + S - bx0, bh = (long long)(-sh[3][0]) + S - by0;
        int st = 0;
        if (sh[4][0] != 0) st = 2;
        else if (bw * bh > kNoAllocMaxBox) st = 1;
        status[0] = st;
        status[1] = bx0;
        status[2] = by0;
        status[3] = st ? 0 : (int)bw;
        status[4] = st ? 0 : (int)bh;
    }
}

// Pass 2 (many CTAs): W_total(x) = sum_k D(x - X_k) at every box node, each node
// summing in ascending k.  A CTA takes 32 x 8 tiles of the box in turn; for each
// chunk of kThreads markers it lists, in ascending order, those whose stencil meets
// the tile (an order-keeping compaction), and every node of the tile then adds the
// listed markers that cover it, so a node only visits markers near its tile.
__global__ void __launch_bounds__(kThreads) noalloc_wtotal_kernel(const double* __restrict__ xy, int n, int kernel,
                                                                  const int* __restrict__ status,
                                                                  double* __restrict__ w) {
    __shared__ int list[kThreads];
    __shared__ int warp_n[kThreads / 32];
    if (status[0] != 0) return;
    const int bx0 = status[1], by0 = status[2], bw = status[3], bh = status[4];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, S = kernel == K_HAT ? 2 : 4;
    const int tiles_x = (bw + kTileW - 1) / kTileW, tiles = tiles_x * ((bh + kTileH - 1) / kTileH);
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int tx0 = bx0 + (t % tiles_x) * kTileW, ty0 = by0 + (t / tiles_x) * kTileH;
        const int x = tx0 + tid % kTileW, y = ty0 + tid / kTileW;
        const bool live = x < bx0 + bw && y < by0 + bh;
        double acc = 0.0;
        for (int c0 = 0; c0 < n; c0 += kThreads) {
            const int k = c0 + tid;
            int hit = 0;
            if (k < n) {
                const int i0 = stencil_origin(kernel, xy[2 * k]), j0 = stencil_origin(kernel, xy[2 * k + 1]);
                hit = i0 <= tx0 + kTileW - 1 && i0 + S - 1 >= tx0 && j0 <= ty0 + kTileH - 1 && j0 + S - 1 >= ty0;
            }
            int v = hit;   // inclusive scan of the hits within the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += u;
            }
            if (lane == 31) warp_n[wid] = v;
            __syncthreads();
            int base = 0, total = 0;
            for (int q = 0; q < kThreads / 32; ++q) {
                base += q < wid ? warp_n[q] : 0;
                total += warp_n[q];
            }
            if (hit) list[base + v - 1] = k;
            __syncthreads();
            if (live) {
                for (int q = 0; q < total; ++q) {
                    const int m = list[q];
                    const double X = xy[2 * m], Y = xy[2 * m + 1];
                    const int i0 = stencil_origin(kernel, X), j0 = stencil_origin(kernel, Y);
                    if (x < i0 || x >= i0 + S || y < j0 || y >= j0 + S) continue;
                    acc += phi_d(kernel, (double)x - X) * phi_d(kernel, (double)y - Y);
                }
            }
            __syncthreads();   // list and warp_n are rewritten by the next chunk
        }
        if (live) w[(size_t)(y - by0) * bw + (x - bx0)] = acc;
    }
}

// Pass 3 (many CTAs): W_sum(k) = sum over the stencil of W_total D and
// lambda_k = 1 / (2 rho_f ds W_sum(k)), rho_f = 1.
__global__ void __launch_bounds__(kThreads) noalloc_lambda_kernel(const double* __restrict__ xy, int n, double ds,
                                                                  int kernel, const int* __restrict__ status,
                                                                  const double* __restrict__ w,
                                                                  double* __restrict__ lam) {
    if (status[0] != 0) return;
    const int bx0 = status[1], by0 = status[2], bw = status[3], S = kernel == K_HAT ? 2 : 4;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < n; k += gridDim.x * kThreads) {
        const double X = xy[2 * k], Y = xy[2 * k + 1];
        const int i0 = stencil_origin(kernel, X), j0 = stencil_origin(kernel, Y);
        double ws = 0.0;
        for (int b = 0; b < S; ++b)
            for (int a = 0; a < S; ++a) {
                const double D = phi_d(kernel, (double)(i0 + a) - X) * phi_d(kernel, (double)(j0 + b) - Y);
                ws += w[(size_t)(j0 + b - by0) * bw + (i0 + a - bx0)] * D;
            }
        lam[k] = 1.0 / (2.0 * 1.0 * ds * ws);
    }
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
    int* status_d = g_status_ptr[dev];
    IBLBM_LAUNCH(noalloc_box_kernel, 1, kThreads, st, xy, n, kernel, nx, ny, status_d);
    IBLBM_LAUNCH(noalloc_wtotal_kernel, kWGrid, kThreads, st, xy, n, kernel, status_d, g_w_ptr[dev]);
    const int lgrid = (n + kThreads - 1) / kThreads;
    IBLBM_LAUNCH(noalloc_lambda_kernel, lgrid, kThreads, st, xy, n, ds, kernel, status_d, g_w_ptr[dev], lambda);
    if (cudaGetLastError() != cudaSuccess) return IBLBM_ERR_CUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, status_d, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    if (status == 1) return IBLBM_ERR_CAPACITY;
    if (status == 2) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
    return IBLBM_OK;
}
