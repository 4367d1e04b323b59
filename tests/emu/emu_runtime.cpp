// Host emulation of the CUDA runtime calls and execution model used by the
// library (TEST INFRASTRUCTURE, see cuda_emu.h).  Blocks run one at a time on
// a pool of host threads, one per CUDA thread; a block that deadlocks aborts.
#include "cuda_emu.h"

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <semaphore>
#include <thread>
#include <vector>

namespace emu {

thread_local ThreadCoord tc;

namespace {

// Generation-counting barrier on futex-backed atomic waits.  A divergent
// barrier leaves its block unfinished; run_block reports that after a timeout.
struct Barrier {
    std::atomic<int> count{0};
    std::atomic<unsigned> gen{0};
    int n = 0;
    void wait(const char*) {
        const unsigned g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) + 1 == n) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_release);
            gen.notify_all();
            return;
        }
        while (gen.load(std::memory_order_acquire) == g) gen.wait(g, std::memory_order_acquire);
    }
};

constexpr int kMaxThreads = 512;

struct Pool {
    // Each worker waits on its own semaphore, so a launch wakes only the
    // threads of its block, not the whole pool.
    std::vector<std::thread> workers;
    std::vector<std::unique_ptr<std::binary_semaphore>> go;
    std::mutex m;
    std::condition_variable cv_done;
    int remaining = 0;
    bool stop = false;
    std::function<void()> body;
    ThreadCoord base;
    Barrier block_bar;
    Barrier warp_bar[kMaxThreads / 32];
    uint64_t warp_buf[kMaxThreads / 32][32];

    Pool() {
        for (int i = 0; i < kMaxThreads; ++i) go.emplace_back(new std::binary_semaphore(0));
        for (int i = 0; i < kMaxThreads; ++i) workers.emplace_back([this, i] { run(i); });
    }
    ~Pool() {
        stop = true;
        for (auto& g : go) g->release();
        for (auto& w : workers) w.join();
    }
    void run(int i) {
        for (;;) {
            go[i]->acquire();
            if (stop) return;
            tc = base;
            tc.tid = make_uint3((unsigned)i, 0, 0);
            body();
            std::lock_guard<std::mutex> lk(m);
            if (--remaining == 0) cv_done.notify_all();
        }
    }
    void run_block(const ThreadCoord& c, int nthreads, const std::function<void()>& f) {
        body = f;
        base = c;
        block_bar.n = nthreads;
        for (int w = 0; w < (nthreads + 31) / 32; ++w) warp_bar[w].n = std::min(32, nthreads - 32 * w);
        {
            std::lock_guard<std::mutex> lk(m);
            remaining = nthreads;
        }
        for (int i = 0; i < nthreads; ++i) go[i]->release();   // release orders the writes above
        std::unique_lock<std::mutex> lk(m);
        // a block that never finishes is a divergent barrier; the limit is generous so that a
        // slow but correct block on a busy host does not trip it
        if (!cv_done.wait_for(lk, std::chrono::seconds(600), [&] { return remaining == 0; })) {
            std::fprintf(stderr, "emu: block did not finish (divergent barrier)\n");
            std::abort();
        }
    }
};

Pool& pool() {
    static Pool* p = new Pool();   // never destroyed: workers live until exit
    return *p;
}

struct Capture {
    std::vector<std::function<void()>> ops;
};
std::map<cudaStream_t, std::shared_ptr<Capture>> g_capturing;
std::mutex g_launch_mu;

void run_now(dim3 grid, dim3 block, const std::function<void()>& body) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    const int nthreads = (int)(block.x * block.y * block.z);
    if (nthreads > kMaxThreads || block.y != 1 || block.z != 1) {
        std::fprintf(stderr, "emu: unsupported block shape\n");
        std::abort();
    }
    for (unsigned bz = 0; bz < grid.z; ++bz)
        for (unsigned by = 0; by < grid.y; ++by)
            for (unsigned bx = 0; bx < grid.x; ++bx) {
                ThreadCoord c;
                c.bid = make_uint3(bx, by, bz);
                c.bdim = block;
                c.gdim = grid;
                pool().run_block(c, nthreads, body);
            }
}

}  // namespace

void syncthreads() { pool().block_bar.wait("block"); }

uint64_t exchange(uint64_t v, int src_lane) {
    Pool& p = pool();
    const int w = (int)(tc.tid.x / 32), lane = (int)(tc.tid.x & 31u);
    p.warp_buf[w][lane] = v;
    p.warp_bar[w].wait("warp");
    const uint64_t r = p.warp_buf[w][src_lane];
    p.warp_bar[w].wait("warp");
    return r;
}

int any(int pred) {
    Pool& p = pool();
    const int w = (int)(tc.tid.x / 32), lane = (int)(tc.tid.x & 31u);
    p.warp_buf[w][lane] = pred ? 1 : 0;
    p.warp_bar[w].wait("warp");
    int r = 0;
    for (int l = 0; l < p.warp_bar[w].n; ++l) r |= (int)p.warp_buf[w][l];
    p.warp_bar[w].wait("warp");
    return r;
}

void launch(dim3 grid, dim3 block, std::function<void()> body, cudaStream_t st) {
    auto it = g_capturing.find(st);
    if (it != g_capturing.end()) {
        it->second->ops.push_back([grid, block, body] { run_now(grid, block, body); });
        return;
    }
    run_now(grid, block, body);
}

unsigned char* dyn_smem() {
    // blocks run one at a time, so one buffer serves every block's dynamic shared memory
    static unsigned char* buf = static_cast<unsigned char*>(std::aligned_alloc(256, 256 * 1024));
    return buf;
}

void yield() { std::this_thread::yield(); }

bool drop_bulk_copies() {
    const char* v = std::getenv("IBLBM_EMU_DROP_BULK_COPIES");
    return v && v[0] == '1';
}

}  // namespace emu

// ---- runtime API --------------------------------------------------------------------------
struct EmuEvent {
    std::chrono::steady_clock::time_point t;
    std::shared_ptr<emu::Capture> cap;   // capture the recording stream was in, if any
};
struct EmuGraph {
    std::vector<std::function<void()>> ops;
};

extern "C" {

cudaError_t cudaMalloc(void** p, size_t n) {
    *p = std::aligned_alloc(256, (n + 255) & ~size_t(255));
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFree(void* p) {
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind) {
    std::memmove(d, s, n);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind, cudaStream_t) {
    std::memmove(d, s, n);
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* d, int v, size_t n, cudaStream_t) {
    std::memset(d, v, n);
    return cudaSuccess;
}
cudaError_t cudaGetDevice(int* d) {
    *d = 0;
    return cudaSuccess;
}
cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr a, int) {
    *v = (a == cudaDevAttrMultiProcessorCount) ? 2 : 1;
    return cudaSuccess;
}
cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int* n, const void*, int, size_t) {
    *n = 1;
    return cudaSuccess;
}
cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessorWithFlags(int* n, const void*, int, size_t, unsigned) {
    *n = 1;
    return cudaSuccess;
}
cudaError_t cudaFuncSetAttribute(const void*, cudaFuncAttribute, int) { return cudaSuccess; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
cudaError_t cudaDeviceSynchronize(void) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned) {
    *s = reinterpret_cast<cudaStream_t>(new char[16]);
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) {
    delete[] reinterpret_cast<char*>(s);
    return cudaSuccess;
}
cudaError_t cudaEventCreate(cudaEvent_t* e) {
    *e = reinterpret_cast<cudaEvent_t>(new EmuEvent());
    return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned) { return cudaEventCreate(e); }
cudaError_t cudaEventDestroy(cudaEvent_t e) {
    delete reinterpret_cast<EmuEvent*>(e);
    return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s) {
    EmuEvent* ev = reinterpret_cast<EmuEvent*>(e);
    ev->t = std::chrono::steady_clock::now();
    auto it = emu::g_capturing.find(s);
    ev->cap = it != emu::g_capturing.end() ? it->second : nullptr;
    return cudaSuccess;
}
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t a, cudaEvent_t b) {
    *ms = std::chrono::duration<float, std::milli>(reinterpret_cast<EmuEvent*>(b)->t -
                                                   reinterpret_cast<EmuEvent*>(a)->t).count();
    return cudaSuccess;
}
cudaError_t cudaStreamWaitEvent(cudaStream_t s, cudaEvent_t e, unsigned) {
    // a stream that waits on an event recorded during a capture joins that capture
    EmuEvent* ev = reinterpret_cast<EmuEvent*>(e);
    if (ev->cap) emu::g_capturing[s] = ev->cap;
    return cudaSuccess;
}
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaGetSymbolAddress(void** p, const void* symbol) {
    *p = const_cast<void*>(symbol);
    return cudaSuccess;
}
cudaError_t cudaStreamBeginCapture(cudaStream_t s, cudaStreamCaptureMode) {
    emu::g_capturing[s] = std::make_shared<emu::Capture>();
    return cudaSuccess;
}
cudaError_t cudaStreamEndCapture(cudaStream_t s, cudaGraph_t* g) {
    auto it = emu::g_capturing.find(s);
    if (it == emu::g_capturing.end()) return cudaErrorIllegalState;
    EmuGraph* eg = new EmuGraph();
    eg->ops = it->second->ops;
    const auto cap = it->second;
    for (auto j = emu::g_capturing.begin(); j != emu::g_capturing.end();)   // joined streams leave too
        j = j->second == cap ? emu::g_capturing.erase(j) : std::next(j);
    *g = reinterpret_cast<cudaGraph_t>(eg);
    return cudaSuccess;
}
cudaError_t cudaGraphInstantiate(cudaGraphExec_t* x, cudaGraph_t g, unsigned long long) {
    EmuGraph* eg = new EmuGraph(*reinterpret_cast<EmuGraph*>(g));
    *x = reinterpret_cast<cudaGraphExec_t>(eg);
    return cudaSuccess;
}
cudaError_t cudaGraphDestroy(cudaGraph_t g) {
    delete reinterpret_cast<EmuGraph*>(g);
    return cudaSuccess;
}
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t x) {
    delete reinterpret_cast<EmuGraph*>(x);
    return cudaSuccess;
}
cudaError_t cudaGraphLaunch(cudaGraphExec_t x, cudaStream_t) {
    for (auto& op : reinterpret_cast<EmuGraph*>(x)->ops) op();
    return cudaSuccess;
}

}  // extern "C"
