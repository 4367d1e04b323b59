// CPU emulation shim for the library's CUDA sources (TEST INFRASTRUCTURE).
//
// Compiling the kernels and the host runtime with g++ and -DIBLBM_EMULATE runs
// every kernel on host threads: one std::thread per CUDA thread of a block,
// blocks one after another, __syncthreads and warp shuffles as barriers with
// a deadlock timeout.  The CUDA runtime calls the library makes are served by
// host memory.  It lets the parity tests exercise the kernel logic without a
// GPU; it is never part of the product library.
#pragma once

#define __shared__ static
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#ifndef __launch_bounds__
#define __launch_bounds__(...)
#endif

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>

namespace emu {
struct ThreadCoord {
    uint3 tid, bid;
    dim3 bdim, gdim;
};
extern thread_local ThreadCoord tc;
void syncthreads();
uint64_t exchange(uint64_t v, int src_lane);   // warp exchange: value of lane src_lane
int any(int pred);
void launch(dim3 grid, dim3 block, std::function<void()> body, cudaStream_t st);
unsigned char* dyn_smem();   // dynamic shared memory of the running block (256 KB)
void yield();
bool drop_bulk_copies();   // IBLBM_EMU_DROP_BULK_COPIES=1: bulk copies never complete (test hook)
}  // namespace emu

#define threadIdx (emu::tc.tid)
#define blockIdx (emu::tc.bid)
#define blockDim (emu::tc.bdim)
#define gridDim (emu::tc.gdim)

inline void __syncthreads() { emu::syncthreads(); }

template <class T>
inline T __ldg(const T* p) { return *p; }
inline long long emu_to_bits_ll(double v) {
    long long b;
    std::memcpy(&b, &v, sizeof(b));
    return b;
}
template <class T>
inline void __stcg(T* p, T v) { *p = v; }
inline long long __double_as_longlong(double v) { return emu_to_bits_ll(v); }
// round-to-nearest FP64 product and sum (the host build targets x86-64 without FMA,
// so these are single roundings as on the device)
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __longlong_as_double(long long v) {
    double d;
    std::memcpy(&d, &v, sizeof(d));
    return d;
}

template <class T>
inline T emu_from_bits(uint64_t b) {
    T v;
    std::memcpy(&v, &b, sizeof(T));
    return v;
}
template <class T>
inline uint64_t emu_to_bits(T v) {
    uint64_t b = 0;
    std::memcpy(&b, &v, sizeof(T));
    return b;
}
template <class T>
inline T __shfl_up_sync(unsigned, T v, unsigned d) {
    const int lane = (int)(threadIdx.x & 31u);
    const int src = lane - (int)d;
    return emu_from_bits<T>(emu::exchange(emu_to_bits(v), src < 0 ? lane : src));
}
template <class T>
inline T __shfl_down_sync(unsigned, T v, unsigned d) {
    const int lane = (int)(threadIdx.x & 31u);
    const int src = lane + (int)d;
    return emu_from_bits<T>(emu::exchange(emu_to_bits(v), src > 31 ? lane : src));
}
template <class T>
inline T __shfl_xor_sync(unsigned, T v, int mask) {
    const int lane = (int)(threadIdx.x & 31u);
    return emu_from_bits<T>(emu::exchange(emu_to_bits(v), lane ^ mask));
}
template <class T>
inline T __shfl_sync(unsigned, T v, int src) {
    return emu_from_bits<T>(emu::exchange(emu_to_bits(v), src & 31));
}
inline int __any_sync(unsigned, int pred) { return emu::any(pred); }
// bytes of {y, x} (x the low word) picked by the four selector nibbles of s
inline unsigned __byte_perm(unsigned x, unsigned y, unsigned s) {
    const unsigned long long v = ((unsigned long long)y << 32) | x;
    unsigned r = 0;
    for (int k = 0; k < 4; ++k) r |= (unsigned)((v >> (8 * ((s >> (4 * k)) & 7u))) & 0xffu) << (8 * k);
    return r;
}
inline void __syncwarp(unsigned = 0xffffffffu) { emu::any(0); }

inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned atomicAdd(unsigned* p, unsigned v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
    return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST);
}
inline void __threadfence() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline unsigned atomicOr(unsigned* p, unsigned v) { return __atomic_fetch_or(p, v, __ATOMIC_SEQ_CST); }

using std::max;
using std::min;

#define IBLBM_LAUNCH(kern, grid, block, stream, ...) \
    emu::launch(dim3(grid), dim3(block), [=]() { kern(__VA_ARGS__); }, (stream))
#define IBLBM_LAUNCH_SMEM(kern, grid, block, smem, stream, ...) \
    emu::launch(dim3(grid), dim3(block), [=]() { kern(__VA_ARGS__); }, (stream))
#define IBLBM_DYNAMIC_SMEM(name) unsigned char* name = emu::dyn_smem()
#define IBLBM_LAUNCH_PDL(kern, grid, block, stream, dependent, ...) \
    emu::launch(dim3(grid), dim3(block), [=]() { kern(__VA_ARGS__); }, (stream))
