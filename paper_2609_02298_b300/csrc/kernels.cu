// Kernels of one IB-LBM step (Sec. 2.1-2.7):
//   ib_kernel      one CTA per body: footprint, post-streaming gather, DF / MDF /
//                  DFC, deterministic spread to a per-body patch, FP64 force and
//                  torque reduction.
//   sc_kernel      fused pull-stream + domain conditions + IB patch + collide,
//                  one warp per row segment of 32 x 16-byte vectors.
//   body_kernel    FP64 rigid-body motion: first half of Eq. 23 and marker motion
//                  before the IB stage, second half with Eq. A3 after it; advances
//                  the step counters.
#include <climits>
#include <type_traits>

#include "async_copy.cuh"
#include "kernels.cuh"

namespace iblbm {

// ------------------------------------------------------------------------------------------
// IB patch lookup shared by stream-collide and the macro export.
// Returns true when a DF/MDF body spread a force onto the node (a DFC patch corrects
// the populations and adds no force).
template <class R>
__device__ __forceinline__ bool add_ib(const CaseDev& C, int x, int y, R (&s)[9], R& Fx, R& Fy) {
    bool forced = false;
    for (int b = 0; b < C.nbodies; ++b) {
        const BodyDev& B = C.bodies[b];
        const int lx = x - B.bx0, ly = y - B.by0;
        if (B.nfp <= 0 || lx < 0 || ly < 0 || lx >= B.bw || ly >= B.bh) continue;
        const int slot = B.node_map[ly * B.bw + lx];
        if (slot < 0) continue;
        const R* p = static_cast<const R*>(B.patch) + (size_t)slot * 9;
        if (B.scheme == SCH_DFC) {
#pragma unroll
            for (int i = 0; i < 9; ++i) s[i] += p[i];
        } else {
            Fx += p[0];
            Fy += p[1];
            forced = true;
        }
    }
    return forced;
}

__device__ __forceinline__ bool row_has_ib(const CaseDev& C, int y, int xa, int xb) {
    bool ib = false;
    for (int b = 0; b < C.nbodies; ++b) {
        const BodyDev& B = C.bodies[b];
        if (B.nfp > 0 && y >= B.by0 && y < B.by0 + B.bh && B.bx0 < xb && B.bx0 + B.bw > xa) ib = true;
    }
    return ib;
}

template <class R>
__device__ __forceinline__ bool bad_density(R rho) {
    return !(rho > R(0) && rho < R(1e30));
}

// Programmatic dependent launch (sm_90 and later): launch_dependents lets the next
// kernel of the stream start once every CTA of this one has issued it; wait blocks
// until the kernel this one depends on has completed and its writes are visible.
// Both return at once for a kernel launched without the dependency.
__device__ __forceinline__ void pdl_trigger() {
#ifndef IBLBM_EMULATE
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait() {
#ifndef IBLBM_EMULATE
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// Thread-block clusters (sm_90 and later): rank of this CTA in its cluster, and a barrier
// of every thread of the cluster with release / acquire semantics at cluster scope (writes
// before it, global memory included, are visible to the cluster's threads after it).  The
// host emulation runs one CTA per cluster.
__device__ __forceinline__ unsigned cluster_rank() {
#ifndef IBLBM_EMULATE
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
#else
    return 0;
#endif
}
__device__ __forceinline__ void cluster_sync_all() {
#ifndef IBLBM_EMULATE
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
#else
    __syncthreads();
#endif
}

// True when the row segment [xseg, xseg + w) of row y lies in the IB region of a body
// of the case (w divides kIbAlign, xseg a multiple of w).
__device__ __forceinline__ bool seg_in_ib(const CaseDev& C, int y, int xseg) {
    for (int b = 0; b < C.nbodies; ++b) {
        const BodyDev& B = C.bodies[b];
        if (B.nfp > 0 && in_ib_region(y, xseg, B.bx0, B.by0, B.bw, B.bh)) return true;
    }
    return false;
}


// ------------------------------------------------------------------------------------------
// Stream-collide of one row segment [xseg, xseg + 32V) of row y, one warp.
template <class S>
struct ScCase {
    using R = typename Traits<S>::R;
    const CaseDev* C;
    const S* src;
    S* dst;
    int nx, ny, pitch, nbodies;
    long long plane;
    bool xper, yper, neu_w, neu_e;
    CollParams<R> P;
    R gfx, gfy;
    bool has_force;
    __device__ __forceinline__ void load(const CaseDev* c) {
        C = c;
        const int parity = (int)(c->step & 1ull);
        src = static_cast<const S*>(c->f[parity]);
        dst = static_cast<S*>(c->f[parity ^ 1]);
        nx = c->nx; ny = c->ny; pitch = c->pitch; nbodies = c->nbodies; plane = c->plane;
        xper = c->bc[SIDE_W] == BC_PER;
        yper = c->bc[SIDE_S] == BC_PER;
        neu_w = c->bc[SIDE_W] == BC_NEU;
        neu_e = c->bc[SIDE_E] == BC_NEU;
        P.load(*c);
        gfx = R(c->gfx);
        gfy = R(c->gfy);
        has_force = c->gfx != 0.0 || c->gfy != 0.0;
    }
};

template <class S, int KIND>
__device__ __forceinline__ void sc_row(const ScCase<S>& K, int y, int xseg, int lane) {
    using R = typename Traits<S>::R;
    constexpr int V = Traits<S>::V;
    const unsigned FULL = 0xffffffffu;
    const CaseDev& C = *K.C;
    const S* __restrict__ src = K.src;
    S* __restrict__ dst = K.dst;
    const int nx = K.nx, ny = K.ny, pitch = K.pitch;
    const long long plane = K.plane;
    const bool xper = K.xper, yper = K.yper;
    const CollParams<R>& P = K.P;
    const R gfx = K.gfx, gfy = K.gfy;
    const int x0 = xseg + lane * V;
    const bool ib = K.nbodies > 0 && row_has_ib(C, y, xseg, xseg + 32 * V);
    bool unstable = false;

    // the first and last rows belong to edge_kernel; side nodes computed here are
    // rewritten by it after this launch
    if (y == 0 || y == ny - 1) return;
    {
        int ym = y - 1, yp = y + 1;
        if (yper) {
            if (ym < 0) ym += ny;
            if (yp >= ny) yp -= ny;
        }
        const bool active = x0 < nx;
        R s[9][V];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sy = ey(i) == 1 ? ym : (ey(i) == -1 ? yp : y);
            const S* row = src + i * plane + (long long)sy * pitch;
            R v[V];
            if (active) {
                ld16(row + x0, v);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) v[k] = R(0);
            }
            if (ex(i) == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) s[i][k] = v[k];
            } else if (ex(i) == 1) {
                R left = __shfl_up_sync(FULL, v[V - 1], 1);
                if (lane == 0) left = x0 > 0 ? ld1(row + x0 - 1) : (xper ? ld1(row + nx - 1) : R(0));
                s[i][0] = left;
#pragma unroll
                for (int k = 1; k < V; ++k) s[i][k] = v[k - 1];
            } else {
                R right = __shfl_down_sync(FULL, v[0], 1);
                if (lane == 31) right = x0 + V < pitch ? ld1(row + x0 + V) : R(0);
#pragma unroll
                for (int k = 0; k < V - 1; ++k) s[i][k] = v[k + 1];
                s[i][V - 1] = right;
            }
        }
        // east / west sides
        const int ke = nx - 1 - x0;                       // position of the east node in this lane
        const bool east_here = ke >= 0 && ke < V;
        const bool east_in_seg = (nx - 1 >= xseg) && (nx - 1 < xseg + 32 * V);
        if (xper) {
            if (east_here) {
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (ex(i) == -1) {
                        const int sy = ey(i) == 1 ? ym : (ey(i) == -1 ? yp : y);
#pragma unroll
                        for (int k = 0; k < V; ++k)
                            if (k == ke) s[i][k] = ld1(src + i * plane + (long long)sy * pitch);
                    }
            }
        } else {
            // zero-gradient east copies node nx-2: same lane, or the previous lane's last node
            R nb[9];
            if (east_in_seg && K.neu_e && ((nx - 1) % V) == 0) {
#pragma unroll
                for (int i = 0; i < 9; ++i) nb[i] = __shfl_up_sync(FULL, s[i][V - 1], 1);
                // node nx-2 opens the previous segment: pull it directly
                if (east_here && lane == 0) pull_node<S, R>(C, src, nx - 2, y, nb);
            }
            if (east_here) {
                if (K.neu_e) {
                    if (ke == 0) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) s[i][0] = nb[i];
                    } else {
#pragma unroll
                        for (int k = 1; k < V; ++k)
                            if (k == ke) {
#pragma unroll
                                for (int i = 0; i < 9; ++i) s[i][k] = s[i][k - 1];
                            }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < V; ++k)
                        if (k == ke) {
                            R t[9];
#pragma unroll
                            for (int i = 0; i < 9; ++i) t[i] = s[i][k];
                            zou_he<R>(SIDE_E, t, R(C.ubc[SIDE_E][0]), R(C.ubc[SIDE_E][1]), (C.wall_bb >> SIDE_E) & 1);
#pragma unroll
                            for (int i = 0; i < 9; ++i) s[i][k] = t[i];
                        }
                }
            }
            if (x0 == 0) {
                if (K.neu_w) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) s[i][0] = s[i][1];
                } else {
                    R t[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) t[i] = s[i][0];
                    zou_he<R>(SIDE_W, t, R(C.ubc[SIDE_W][0]), R(C.ubc[SIDE_W][1]), (C.wall_bb >> SIDE_W) & 1);
#pragma unroll
                    for (int i = 0; i < 9; ++i) s[i][0] = t[i];
                }
            }
        }
        // IB patch, collision
#pragma unroll
        for (int k = 0; k < V; ++k) {
            R t[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) t[i] = s[i][k];
            R Fx = gfx, Fy = gfy;
            if (ib && x0 + k < nx) add_ib<R>(C, x0 + k, y, t, Fx, Fy);
            const R rho = (ib || K.has_force) ? collide<R, KIND>(P, t, Fx, Fy) : collide<R, KIND, false>(P, t, Fx, Fy);
            if (x0 + k < nx) unstable |= bad_density(rho);
#pragma unroll
            for (int i = 0; i < 9; ++i) s[i][k] = t[i];
        }
        if (active) {
            if (x0 + V <= nx) {
#pragma unroll
                for (int i = 0; i < 9; ++i) st16(dst + i * plane + (long long)y * pitch + x0, s[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 9; ++i)
#pragma unroll
                    for (int k = 0; k < V; ++k)
                        if (x0 + k < nx) st1(dst + i * plane + (long long)y * pitch + x0 + k, s[i][k]);
            }
        }
    }
    if (__any_sync(FULL, unstable) && lane == 0) atomicOr(const_cast<unsigned*>(&C.status), STAT_UNSTABLE);
}

// Each warp takes a contiguous range of jobs (row segments), so the case
// changes rarely; its parameters stay in registers across jobs.
// Resident CTAs per SM each specialisation is compiled for (its register budget
// is 65536 / (256 x this)); chosen from -Xptxas -v so that no variant spills.
template <class S, int KIND> struct ScMinBlocks { static constexpr int value = 2; };
template <> struct ScMinBlocks<double, COL_BGK> { static constexpr int value = 1; };
template <> struct ScMinBlocks<double, COL_TRT> { static constexpr int value = 1; };
template <> struct ScMinBlocks<double, COL_CM> { static constexpr int value = 1; };
template <> struct ScMinBlocks<double, COL_NONE> { static constexpr int value = 1; };
template <> struct ScMinBlocks<double, -1> { static constexpr int value = 1; };
template <int KIND> struct ScMinBlocks<__half, KIND> { static constexpr int value = 1; };

template <class S, int KIND>
__global__ void __launch_bounds__(kThreads, (ScMinBlocks<S, KIND>::value)) sc_kernel(ScLaunch L, long long jobs) {
    constexpr int V = Traits<S>::V;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kThreads) >> 5;
    const long long j0 = jobs * gw / nw, j1 = jobs * (gw + 1) / nw;
    ScCase<S> K;
    long long c_lo = 0, c_hi = 0;
    int nseg = 1, y = 0, seg = 0;
    for (long long job = j0; job < j1; ++job) {
        if (job >= c_hi || job < c_lo) {
            int lo = 0, hi = L.ncases - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (L.job_off[mid] <= job) lo = mid; else hi = mid - 1;
            }
            c_lo = L.job_off[lo];
            c_hi = L.job_off[lo + 1];
            K.load(L.cases[lo]);
            nseg = (K.nx + 32 * V - 1) / (32 * V);
            const long long local = job - c_lo;
            y = (int)(local / nseg);
            seg = (int)(local % nseg);
        }
        sc_row<S, KIND>(K, y, seg * 32 * V, lane);
        if (++seg == nseg) {
            seg = 0;
            ++y;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Stream-collide, NPT nodes per lane: a warp handles NPT chunks of 32 consecutive
// nodes of a row (x = xseg + 32 j + lane) and pulls each population with a plain
// coalesced (possibly one-element unaligned) load.  Only interior nodes are
// computed here (1 <= x <= nx-2, 1 <= y <= ny-2): lattice-edge nodes go to
// edge_kernel, so the warp path carries no wrap or boundary logic (measured on
// B300: a boundary branch inside the sweep costs a third of the HBM rate).
// 32-bit element offsets with per-population constants; the Guo term only on rows
// that carry a force.
// KEEP: the stores carry an L2 evict-last hint (IB-region segments, st1_keep); EVF: the
// loads an L2 evict-first hint (the sweep beside the IB stage, ld1_sweep_ef).
template <class S, int KIND, int NPT, bool KEEP = false, bool EVF = false>
__device__ __forceinline__ void sc_row_scalar(const ScCase<S>& K, int y, int xseg, int lane) {
    using R = typename Traits<S>::R;
    const CaseDev& C = *K.C;
    const S* __restrict__ src = K.src;
    S* __restrict__ dst = K.dst;
    const int nx = K.nx, ny = K.ny, pitch = K.pitch, plane = (int)K.plane;
    if (y == 0 || y == ny - 1) return;
    const bool ib = K.nbodies > 0 && row_has_ib(C, y, xseg, xseg + 32 * NPT);
    const bool forced = ib || K.has_force;
    // pull offset of population i relative to the node: i plane - e_iy pitch - e_ix
    int koff[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) koff[i] = i * plane - ey(i) * pitch - ex(i);
    const int row = y * pitch;
    bool unstable = false;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int x = xseg + 32 * j + lane;
        if (x >= 1 && x < nx - 1) {
            R s[9];
            const int a = row + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if constexpr (EVF) s[i] = ld1_sweep_ef(src + (a + koff[i]));
                else s[i] = ld1_sweep(src + (a + koff[i]));
            }
            R rho;
            if (forced) {
                R Fx = K.gfx, Fy = K.gfy;
                if (ib) add_ib<R>(C, x, y, s, Fx, Fy);
                rho = collide<R, KIND>(K.P, s, Fx, Fy);
            } else {
                rho = collide<R, KIND, false>(K.P, s, R(0), R(0));
            }
            unstable |= bad_density(rho);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if constexpr (KEEP) st1_keep(dst + (a + i * plane), s[i]);
                else st1_sweep(dst + (a + i * plane), s[i]);
            }
        }
    }
    if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(const_cast<unsigned*>(&C.status), STAT_UNSTABLE);
}

// The tail CTAs' form of sc_row_scalar (KEEP stores) in two parts: row_pre takes the pulls
// and the segment's IB decision before the wait for the IB stage (they read nothing that
// stage writes), row_post the patch, collision and stores after it.  The expressions are
// those of sc_row_scalar, so the results are too.
template <class S, int NPT> struct RowPre {
    typename Traits<S>::R s[NPT][9];
    bool ib;
};
template <class S, int NPT>
__device__ __forceinline__ void row_pre(const ScCase<S>& K, int y, int xseg, int lane, RowPre<S, NPT>& P) {
    const int nx = K.nx, ny = K.ny, pitch = K.pitch, plane = (int)K.plane;
    P.ib = false;
    if (y == 0 || y == ny - 1) return;
    P.ib = K.nbodies > 0 && row_has_ib(*K.C, y, xseg, xseg + 32 * NPT);
    int koff[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) koff[i] = i * plane - ey(i) * pitch - ex(i);
    const int row = y * pitch;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int x = xseg + 32 * j + lane;
        if (x >= 1 && x < nx - 1) {
            const int a = row + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) P.s[j][i] = ld1_sweep(K.src + (a + koff[i]));
        }
    }
}
template <class S, int KIND, int NPT>
__device__ __forceinline__ void row_post(const ScCase<S>& K, int y, int xseg, int lane, RowPre<S, NPT>& P) {
    using R = typename Traits<S>::R;
    const CaseDev& C = *K.C;
    S* __restrict__ dst = K.dst;
    const int nx = K.nx, ny = K.ny, pitch = K.pitch, plane = (int)K.plane;
    if (y == 0 || y == ny - 1) return;
    const bool ib = P.ib;
    const bool forced = ib || K.has_force;
    const int row = y * pitch;
    bool unstable = false;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const int x = xseg + 32 * j + lane;
        if (x >= 1 && x < nx - 1) {
            R* s = P.s[j];
            const int a = row + x;
            R rho;
            if (forced) {
                R Fx = K.gfx, Fy = K.gfy;
                if (ib) add_ib<R>(C, x, y, P.s[j], Fx, Fy);
                rho = collide<R, KIND>(K.P, P.s[j], Fx, Fy);
            } else {
                rho = collide<R, KIND, false>(K.P, P.s[j], R(0), R(0));
            }
            unstable |= bad_density(rho);
#pragma unroll
            for (int i = 0; i < 9; ++i) st1_keep(dst + (a + i * plane), s[i]);
        }
    }
    if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(const_cast<unsigned*>(&C.status), STAT_UNSTABLE);
}

// FP16 storage, NP pairs of adjacent nodes per lane: a warp handles NP chunks of 64
// nodes of a row, lane l the pair (x0, x0 + 1), x0 = xseg + 64 j + 2 l.  Each
// population is one aligned 32-bit load of the source row's pair at x0 (two nodes, half
// the load instructions of one node per lane); the pull from x - 1 or x + 1 takes one
// half from the neighbouring lane's word (warp shuffle) and the edge lanes load the
// missing word.  Nodes are unpacked, collided and rounded exactly as in sc_row_scalar,
// so the results are bit for bit those of the one-node-per-lane sweep.
template <int KIND, int NP>
__device__ __forceinline__ void sc_row_pair(const ScCase<__half>& K, int y, int xseg, int lane) {
    using R = float;
    const CaseDev& C = *K.C;
    const __half* __restrict__ src = K.src;
    __half* __restrict__ dst = K.dst;
    const int nx = K.nx, ny = K.ny, pitch = K.pitch, plane = (int)K.plane;
    if (y == 0 || y == ny - 1) return;
    const bool ib = K.nbodies > 0 && row_has_ib(C, y, xseg, xseg + 64 * NP);
    const bool forced = ib || K.has_force;
    const int row = y * pitch;
    bool unstable = false;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int x0 = xseg + 64 * j + 2 * lane;
        const bool inrow = x0 < pitch;   // the pair lies in the padded row (pitch is even)
        R s0[9], s1[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const __half* sr = src + (row + i * plane - ey(i) * pitch);   // source row of population i
            const unsigned a = inrow ? ld2h_sweep(sr + x0) : 0u;
            unsigned v;
            if (ex(i) == 0) {
                v = a;
            } else if (ex(i) == 1) {        // the pair pulls from x0 - 1, x0
                unsigned p = __shfl_up_sync(0xffffffffu, a, 1);
                if (lane == 0) p = (inrow && x0 >= 2) ? ld2h_sweep(sr + x0 - 2) : 0u;
                v = __byte_perm(p, a, 0x5432);
            } else {                        // from x0 + 1, x0 + 2
                unsigned q = __shfl_down_sync(0xffffffffu, a, 1);
                if (lane == 31) q = (x0 + 2 < pitch) ? ld2h_sweep(sr + x0 + 2) : 0u;
                v = __byte_perm(a, q, 0x5432);
            }
            const float2 f = unpack2h(v);
            s0[i] = f.x;
            s1[i] = f.y;
        }
        const bool w0 = x0 >= 1 && x0 < nx - 1, w1 = x0 + 1 < nx - 1;
        if (forced) {
            if (w0) {
                R Fx = K.gfx, Fy = K.gfy;
                if (ib) add_ib<R>(C, x0, y, s0, Fx, Fy);
                unstable |= bad_density(collide<R, KIND>(K.P, s0, Fx, Fy));
            }
            if (w1) {
                R Fx = K.gfx, Fy = K.gfy;
                if (ib) add_ib<R>(C, x0 + 1, y, s1, Fx, Fy);
                unstable |= bad_density(collide<R, KIND>(K.P, s1, Fx, Fy));
            }
        } else {
            if (w0) unstable |= bad_density(collide<R, KIND, false>(K.P, s0, R(0), R(0)));
            if (w1) unstable |= bad_density(collide<R, KIND, false>(K.P, s1, R(0), R(0)));
        }
        __half* d = dst + (row + x0);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (w0 && w1) {
                st2h(d + i * plane, s0[i], s1[i]);
            } else {
                if (w0) st1(d + i * plane, s0[i]);
                if (w1) st1(d + i * plane + 1, s1[i]);
            }
        }
    }
    if (__any_sync(0xffffffffu, unstable) && lane == 0) atomicOr(const_cast<unsigned*>(&C.status), STAT_UNSTABLE);
}

template <class S, int KIND, int NPT> struct ScScalarMinBlocks { static constexpr int value = 4; };
template <int KIND, int NPT> struct ScScalarMinBlocks<double, KIND, NPT> { static constexpr int value = 2; };

// Dense job order: warp w takes jobs w, w + W, w + 2W, ... (W warps in the grid),
// so the warps resident at any moment sweep one compact window of each plane;
// measured on B300 this beats one contiguous job range per warp by ~10% of HBM.
// (Taking jobs from a global counter instead, two jobs per atomic, ran 1.7-2.5x
// slower: the counter's atomics serialise.)  All CTAs of a launch must be resident
// together for the split to balance, which the host arranges when the IB stage runs
// beside the sweep (the grid leaves its SMs free).
// Row segment of the scalar variants: NPT nodes per lane, or NPT adjacent pairs per lane
// for FP16 storage (sc_row_pair).
template <class S, int NPT> struct ScSeg { static constexpr int value = 32 * NPT; };
template <int NPT> struct ScSeg<__half, NPT> { static constexpr int value = 64 * NPT; };
template <class S, int KIND, int NPT, bool KEEP = false, bool EVF = false>
__device__ __forceinline__ void sc_row_nodes(const ScCase<S>& K, int y, int xseg, int lane) {
    if constexpr (std::is_same<S, __half>::value) sc_row_pair<KIND, NPT>(K, y, xseg, lane);
    else sc_row_scalar<S, KIND, NPT, KEEP, EVF>(K, y, xseg, lane);
}

// Lattice-edge node e of a case (rows 0 and ny-1, columns 0 and nx-1): pull with wrap and
// domain conditions (post_stream_node), IB patch, collision with the case's own operator,
// store.  C is the case record (possibly a shared-memory copy), gc the case in global
// memory (status flags).  Edge node e: e < nx -> (e, 0); e < 2nx -> (e - nx, ny - 1) when
// ny > 1; then columns 0 and nx-1 of rows 1..ny-2, alternating.
// In two parts, so that the tail CTAs can pull before they wait for the IB stage.
template <class S>
__device__ __forceinline__ void edge_pre(const CaseDev& C, const ScCase<S>& K, int e, int& x, int& y,
                                         typename Traits<S>::R (&s)[9]) {
    using R = typename Traits<S>::R;
    const int nx = K.nx, ny = K.ny;
    if (e < nx) {
        x = e; y = 0;
    } else if (ny > 1 && e < 2 * nx) {
        x = e - nx; y = ny - 1;
    } else {
        const int r = e - (ny > 1 ? 2 * nx : nx);
        if (nx > 1) { y = 1 + (r >> 1); x = (r & 1) ? nx - 1 : 0; }
        else { y = 1 + r; x = 0; }
    }
    post_stream_node<S, R>(C, K.src, x, y, s);
}
template <class S>
__device__ __forceinline__ void edge_post(const CaseDev& C, const ScCase<S>& K, int x, int y, bool noib,
                                          const CaseDev* gc, typename Traits<S>::R (&s)[9]) {
    using R = typename Traits<S>::R;
    R Fx = K.gfx, Fy = K.gfy;
    if (K.nbodies > 0 && !noib) add_ib<R>(C, x, y, s, Fx, Fy);
    const R rho = collide<R, -1>(K.P, s, Fx, Fy);
    if (bad_density(rho)) atomicOr(const_cast<unsigned*>(&gc->status), STAT_UNSTABLE);
    S* d = K.dst + ((long long)y * K.pitch + x);
#pragma unroll
    for (int i = 0; i < 9; ++i) st1(d + i * K.plane, s[i]);
}
template <class S>
__device__ __forceinline__ void edge_node(const CaseDev& C, const ScCase<S>& K, int e, bool noib, const CaseDev* gc) {
    typename Traits<S>::R s[9];
    int x, y;
    edge_pre<S>(C, K, e, x, y, s);
    edge_post<S>(C, K, x, y, noib, gc, s);
}

// Last CTA of a launch to finish ends the step: advances the step counter of every case
// (every read of the counters in the step is done by then); done[0] counts finished CTAs
// and is reset for the next step.
__device__ __forceinline__ void end_step_if_last(unsigned* done, CaseDev** cases, int ncases) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (last) {   // (the whole CTA: one counter per thread)
        __threadfence();
        for (int c = threadIdx.x; c < ncases; c += blockDim.x) cases[c]->step += 1ull;
        if (threadIdx.x == 0) done[0] = 0u;
    }
}

// Work of the tail CTAs of a SC_SKIP_IB launch (warp w of nw): once the IB stage has
// ended, the listed IB-region segments, then the lattice-edge chunks, one job per warp in
// turn.
template <class S, int KIND, int NPT>
__device__ __forceinline__ void sc_tail(const ScLaunch& L, int w, int nw, int lane) {
    using R = typename Traits<S>::R;
    constexpr bool SPLIT = !std::is_same<S, __half>::value;   // (FP16 pairs: sc_row_pair)
    ScCase<S> K;
    const CaseDev* cur = nullptr;
    const long long njobs = L.nlist + L.nechunks;
    // the first job's reads that the IB stage leaves alone (case record, pulls, the segment's
    // IB decision) go out before the wait
    RowPre<S, NPT> P;
    R es[9];
    int4 e0 = make_int4(0, 0, 0, 0);
    int ex0 = 0, ey0 = 0;
    bool live0 = false;
    if (w < njobs) {
        if (w < L.nlist) {
            e0 = L.list[w];
            cur = L.cases[e0.x];
            K.load(cur);
            if constexpr (SPLIT) row_pre<S, NPT>(K, e0.y, e0.z, lane, P);
        } else {
            const EdgeChunk ch = L.echunks[w - L.nlist];
            cur = L.ecases[ch.c];
            K.load(cur);
            live0 = ch.first + lane < ch.end;
            if (live0) edge_pre<S>(*cur, K, ch.first + lane, ex0, ey0, es);
        }
    }
    if (L.pdl & PDL_DEPENDENT) pdl_wait();   // the IB stage has ended, its patches are visible
    if (w < njobs) {
        if (w < L.nlist) {
            if constexpr (SPLIT) row_post<S, KIND, NPT>(K, e0.y, e0.z, lane, P);
            else sc_row_nodes<S, KIND, NPT, true>(K, e0.y, e0.z, lane);
        } else if (live0) {
            edge_post<S>(*cur, K, ex0, ey0, false, cur, es);
        }
    }
    for (long long j = w + nw; j < njobs; j += nw) {
        if (j < L.nlist) {
            const int4 e = L.list[j];
            const CaseDev* c = L.cases[e.x];
            if (c != cur) {
                K.load(c);
                cur = c;
            }
            sc_row_nodes<S, KIND, NPT, true>(K, e.y, e.z, lane);
        } else {
            const EdgeChunk ch = L.echunks[j - L.nlist];
            const CaseDev* c = L.ecases[ch.c];
            if (c != cur) {
                K.load(c);
                cur = c;
            }
            const int e = ch.first + lane;
            if (e < ch.end) edge_node<S>(*c, K, e, false, c);
        }
    }
}

// MODE (SC_MODE_*): SKIP, the launch beside the IB stage (segments in IB regions left out,
// programmatic dependent launch) with tail CTAs; TAIL, every segment plus tail CTAs for the
// lattice edges and the step end; the plain whole-lattice launch is compiled without either.
template <class S, int KIND, int NPT, int MODE>
__global__ void __launch_bounds__(kThreads, (ScScalarMinBlocks<S, KIND, NPT>::value))
    sc_kernel_scalar(ScLaunch L, long long jobs) {
    constexpr int kSegW = ScSeg<S, NPT>::value;
    constexpr bool SKIP = MODE == SC_MODE_SKIP, TAIL = MODE != SC_MODE_PLAIN;
    if (SKIP && (L.pdl & PDL_TRIGGER)) pdl_trigger();
    const int lane = threadIdx.x & 31;
    // with tail CTAs the segments of the first phase are split over the other CTAs
    const int nblk = TAIL ? (int)gridDim.x - L.tail_ctas : (int)gridDim.x;
    const int wpc = (int)blockDim.x >> 5;
    if (TAIL && (int)blockIdx.x >= nblk) {
        sc_tail<S, KIND, NPT>(L, ((int)blockIdx.x - nblk) * wpc + ((int)threadIdx.x >> 5), L.tail_ctas * wpc, lane);
        if (L.done) end_step_if_last(L.done, L.count_cases, L.ncount);
        return;
    }
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = (long long)nblk * wpc;
    ScCase<S> K;
    long long c_lo = 0, c_hi = 0;
    int nseg = 1;
    for (long long job = gw; job < jobs; job += nw) {
        if (job >= c_hi || job < c_lo) {
            int lo = 0, hi = L.ncases - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (L.job_off[mid] <= job) lo = mid; else hi = mid - 1;
            }
            c_lo = L.job_off[lo];
            c_hi = L.job_off[lo + 1];
            K.load(L.cases[lo]);
            nseg = (K.nx + kSegW - 1) / kSegW;
        }
        const int local = (int)(job - c_lo);   // < ny * nseg
        const int y = local / nseg;
        const int xseg = (local - y * nseg) * kSegW;
        if (SKIP && K.nbodies > 0 && seg_in_ib(*K.C, y, xseg)) continue;
        sc_row_nodes<S, KIND, NPT, false, SKIP>(K, y, xseg, lane);
    }
    if (SKIP && L.tail_ctas == 0 && (L.pdl & PDL_DEPENDENT)) pdl_wait();
    if (TAIL && L.done) end_step_if_last(L.done, L.count_cases, L.ncount);
}

// The SC_LIST phase: the listed segments (IB regions), warp w taking entries w, w + W, ...
template <class S, int KIND, int NPT>
__global__ void __launch_bounds__(kThreads, (ScScalarMinBlocks<S, KIND, NPT>::value))
    sc_kernel_list(ScLaunch L, long long jobs) {
    if (L.pdl & PDL_TRIGGER) pdl_trigger();
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    ScCase<S> K;
    int cur = -1;
    for (long long job = gw; job < jobs; job += nw) {
        const int4 e = L.list[job];
        if (e.x != cur) {
            K.load(L.cases[e.x]);
            cur = e.x;
        }
        sc_row_nodes<S, KIND, NPT>(K, e.y, e.z, lane);
    }
}

// ------------------------------------------------------------------------------------------
// Lattice-edge nodes (rows 0 and ny-1, columns 0 and nx-1) of every case of one
// storage type, one node per thread, one CTA per chunk of 256 edge nodes of one
// case (chunk table built on the host): pull with wrap and domain conditions
// (post_stream_node), IB patch, collision with the case's own operator, store.
// Runs after the stream-collide launches of the step and is the only writer of
// these nodes' results (a variant that also wrote them is overwritten); in the
// overlap order with one storage type the last stream-collide launch does this work
// itself (edge_node in its tail).
__host__ __device__ inline long long edge_count(int nx, int ny) {
    const long long rows = (long long)nx * (ny > 1 ? 2 : 1);
    const long long cols = ny > 2 ? (long long)(ny - 2) * (nx > 1 ? 2 : 1) : 0;
    return rows + cols;
}

template <class S>
__global__ void __launch_bounds__(kThreads) edge_kernel(EdgeLaunch L) {
    // one CTA per 256 edge nodes of one case; the case record is staged in shared
    // memory so the boundary logic reads it without global round trips
    __shared__ __align__(16) CaseDev sc;
    const EdgeChunk ch = L.chunks[blockIdx.x];
    const CaseDev* gc = L.cases[ch.c];
    {
        static_assert(sizeof(CaseDev) % 4 == 0, "case record copied as words");
        const int* from = reinterpret_cast<const int*>(gc);
        int* to = reinterpret_cast<int*>(&sc);
        for (int w = threadIdx.x; w < (int)(sizeof(CaseDev) / 4); w += blockDim.x) to[w] = from[w];
    }
    __syncthreads();
    ScCase<S> K;
    K.load(&sc);
    const int e = ch.first + (int)threadIdx.x;
    if (e < ch.end) edge_node<S>(sc, K, e, L.noib != 0, gc);
    if (L.pdl & PDL_DEPENDENT) pdl_wait();   // the launch before this one has finished too
    if (L.count_cases) end_step_if_last(L.done, L.count_cases, L.ncount);
}

// ------------------------------------------------------------------------------------------
// Stream-collide with bulk-staged sources (SC_BULK).  A job is a tile of TW nodes
// of one row; its nine source rows (row y - e_iy of plane i, columns x0 - H ..
// x0 + TW + H, H = one 16-byte halo) arrive in shared memory by cp.async.bulk.
// Warp-specialised pipeline over NST stages: one producer warp fills stage k and
// signals full[k] through the transaction count; eight consumer warps compute the
// tile from shared memory (one load per population at a constant offset) and
// release the stage on empty[k].  The copy engine keeps several tiles per CTA in
// flight without holding registers, which a pull-streaming sweep needs to cover
// HBM latency.  Lattice-edge nodes and the first and last rows take the general
// path (global pulls with the domain conditions), as in the other variants.
template <class S> struct BulkCfg;
template <> struct BulkCfg<float> { static constexpr int NPT = 2, NST = 6, MINB = 2; };
// FP16: four shallow pipelines per SM (a CTA's 56 registers and 38 KB of stages) measured 5 %
// faster than two deep ones (8 stages, 96 registers): the sweep is short of warps, not of stages
template <> struct BulkCfg<__half> { static constexpr int NPT = 2, NST = 4, MINB = 4; };
template <> struct BulkCfg<double> { static constexpr int NPT = 1, NST = 6, MINB = 2; };
constexpr int kBulkConsumers = kThreads;          // eight consumer warps
constexpr int kBulkThreads = kThreads + 32;       // plus one producer warp
struct BulkDesc {                                 // tile of a stage, written by the producer
    int c, y, x0, flags;
};
enum : int { BULK_STAGED = 1, BULK_INTERIOR = 2, BULK_IB = 4 };
template <class S> struct BulkGeom {
    static constexpr int NST = BulkCfg<S>::NST;
    static constexpr int H = 16 / (int)sizeof(S);
    static constexpr int TW = kBulkConsumers * BulkCfg<S>::NPT;
    static constexpr int RS = TW + 2 * H;                           // elements per staged row
    static constexpr int STAGE = 9 * RS * (int)sizeof(S);           // bytes per stage
    static constexpr int HDR = 16 * NST + 16 * NST + 16;            // full + empty barriers, descriptors, flag
    static constexpr int BAR = (HDR + 127) / 128 * 128;             // header, keeps stages aligned
    static constexpr int SMEM = BAR + NST * STAGE;
    static_assert((RS * (int)sizeof(S)) % 16 == 0, "staged rows must stay 16-byte aligned");
    static_assert(SMEM <= 226 * 1024 / BulkCfg<S>::MINB, "the CTAs per SM must fit");
};
#ifndef IBLBM_EMULATE
constexpr long kBulkSpinLimit = 1L << 22;   // polls of an mbarrier before the kernel gives up
#else
constexpr long kBulkSpinLimit = 1L << 16;   // host emulation: each poll yields the thread
#endif
// Polls of the consumers' wait for a staged tile (kBulkSpinLimit unless lowered through
// iblbm_test_set_consumer_poll_limit, which exists to exercise the give-up path).  The
// producer's waits, including its drain of copies still in flight, keep kBulkSpinLimit.
__device__ long g_consumer_poll_limit = kBulkSpinLimit;

// Wait for a phase, giving up after `limit` polls or as soon as `abort` is raised.
__device__ __forceinline__ bool bar_wait_unless(uint64_t* bar, unsigned parity, long limit, volatile int& abort) {
    for (long it = 0; it < limit; ++it) {
        if (bar_test(bar, parity)) return true;
        if (abort) return false;
    }
    return false;
}

__device__ __forceinline__ double lds1(const double* p) { return *p; }
__device__ __forceinline__ float lds1(const float* p) { return *p; }
__device__ __forceinline__ float lds1(const __half* p) { return __half2float(*p); }

// Case index, row and first column of tile `job`.
template <int TW>
__device__ __forceinline__ int bulk_locate(const ScLaunch& L, long long job, int& y, int& x0) {
    int lo = 0, hi = L.ncases - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.job_off[mid] <= job) lo = mid; else hi = mid - 1;
    }
    const CaseDev& C = *L.cases[lo];
    const int nseg = (C.nx + TW - 1) / TW;
    const long long local = job - L.job_off[lo];
    y = (int)(local / nseg);
    x0 = (int)(local % nseg) * TW;
    return lo;
}

// Producer's position in the job list with the current case's fields cached, so
// that a tile costs no global loads beyond its copies.  The IB flag uses the union
// of the case's body boxes (conservative: add_ib checks each node exactly).
struct BulkCursor {
    int c, y, seg, nseg, nx, ny, pitch;
    long long plane, end;
    const void* src;
    int iy0, iy1, ix0, ix1;
};

template <int TW>
__device__ __forceinline__ void cursor_load(const ScLaunch& L, BulkCursor& u, int c, long long job) {
    const CaseDev& C = *L.cases[c];
    u.c = c;
    u.nx = C.nx;
    u.ny = C.ny;
    u.pitch = C.pitch;
    u.plane = C.plane;
    u.nseg = (C.nx + TW - 1) / TW;
    u.end = L.job_off[c + 1];
    const long long local = job - L.job_off[c];
    u.y = (int)(local / u.nseg);
    u.seg = (int)(local % u.nseg);
    u.src = C.f[(int)(C.step & 1ull)];
    u.iy0 = INT_MAX; u.iy1 = INT_MIN; u.ix0 = INT_MAX; u.ix1 = INT_MIN;
    for (int b = 0; b < C.nbodies; ++b) {
        const BodyDev& B = C.bodies[b];
        if (B.nfp <= 0) continue;
        u.iy0 = min(u.iy0, B.by0); u.iy1 = max(u.iy1, B.by0 + B.bh);
        u.ix0 = min(u.ix0, B.bx0); u.ix1 = max(u.ix1, B.bx0 + B.bw);
    }
}

// Describe the cursor's tile in `desc` and start its nine row copies into `st`.
template <class S>
__device__ __forceinline__ void bulk_issue(const BulkCursor& u, S* st, uint64_t* full, BulkDesc* desc) {
    using G = BulkGeom<S>;
    const int y = u.y, x0 = u.seg * G::TW;
    const bool staged = y > 0 && y < u.ny - 1;
    const bool interior = staged && x0 > 0 && x0 + G::TW < u.nx - 1;
    const bool ib = y >= u.iy0 && y < u.iy1 && u.ix0 < x0 + G::TW && u.ix1 > x0;
    desc->c = u.c;
    desc->y = y;
    desc->x0 = x0;
    desc->flags = (staged ? BULK_STAGED : 0) | (interior ? BULK_INTERIOR : 0) | (ib ? BULK_IB : 0);
    if (!staged) {   // general path: nothing to copy
        bar_arrive_tx(full, 0);
        return;
    }
    const S* src = static_cast<const S*>(u.src);
    const int xs = max(x0 - G::H, 0), xe = min(x0 + G::TW + G::H, u.pitch);
    const unsigned bytes = (unsigned)((xe - xs) * (int)sizeof(S));
    bar_arrive_tx(full, 9u * bytes);
#pragma unroll
    for (int i = 0; i < 9; ++i)
        bulk_g2s(st + i * G::RS + (xs - x0 + G::H), src + i * u.plane + (long long)(y - ey(i)) * u.pitch + xs, bytes,
                 full);
}

__device__ __forceinline__ void stg1(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stg1(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void stg1(__half* p, float v) { __stcg(p, __float2half_rn(v)); }

// One node of a staged tile: pull from the stage, IB patch, collision, streaming store.
template <class S, int KIND, bool FORCED>
__device__ __forceinline__ bool bulk_node(const ScCase<S>& K, const S* b, S* d, int x, int y, bool ib) {
    using R = typename Traits<S>::R;
    R s[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) s[i] = lds1(b + i * BulkGeom<S>::RS - ex(i));
    R rho;
    if (FORCED) {
        R Fx = K.gfx, Fy = K.gfy;
        if (ib) add_ib<R>(*K.C, x, y, s, Fx, Fy);
        rho = collide<R, KIND>(K.P, s, Fx, Fy);
    } else {
        rho = collide<R, KIND, false>(K.P, s, R(0), R(0));
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) stg1(d + i * K.plane, s[i]);
    return bad_density(rho);
}

// All interior nodes of a tile: interior tiles take the stage without checks;
// staged tiles touching a side skip that side's edge node; edge rows hold no
// interior nodes (edge_kernel computes every lattice-edge node).
template <class S, int KIND, bool FORCED>
__device__ __forceinline__ bool bulk_tile(const ScCase<S>& K, const S* st, S* d, int x0, int y, int flags, int tid) {
    constexpr int NPT = BulkCfg<S>::NPT;
    const bool ib = (flags & BULK_IB) != 0;
    bool unstable = false;
    if (flags & BULK_INTERIOR) {
#pragma unroll
        for (int j = 0; j < NPT; ++j)
            unstable |= bulk_node<S, KIND, FORCED>(K, st + kBulkConsumers * j, d + kBulkConsumers * j,
                                                   x0 + tid + kBulkConsumers * j, y, ib);
    } else if (flags & BULK_STAGED) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const int x = x0 + tid + kBulkConsumers * j;
            if (x > 0 && x < K.nx - 1)
                unstable |= bulk_node<S, KIND, FORCED>(K, st + kBulkConsumers * j, d + kBulkConsumers * j, x, y, ib);
        }
    }
    return unstable;
}

template <class S, int KIND>
__global__ void __launch_bounds__(kBulkThreads, (BulkCfg<S>::MINB)) sc_kernel_bulk(ScLaunch L, long long jobs) {
    using G = BulkGeom<S>;
    constexpr int NST = G::NST, TW = G::TW, RS = G::RS, H = G::H;
    IBLBM_DYNAMIC_SMEM(smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NST;
    BulkDesc* desc = reinterpret_cast<BulkDesc*>(smem + 16 * NST);
    volatile int& abort_flag = *reinterpret_cast<int*>(smem + 32 * NST);
    S* stages = reinterpret_cast<S*>(smem + G::BAR);
    const int tid = threadIdx.x;
    const long long j0 = jobs * blockIdx.x / gridDim.x, j1 = jobs * (blockIdx.x + 1) / gridDim.x;
    if (tid == 0) {
        for (int k = 0; k < NST; ++k) {
            bar_init(&full[k], 1);
            bar_init(&empty[k], kBulkConsumers / 32);
        }
        fence_bar_init();
        abort_flag = 0;
    }
    __syncthreads();

    if (tid >= kBulkConsumers) {
        // producer warp: lane 0 streams the CTA's tiles through the stages
        if (tid == kBulkConsumers && j0 < j1) {
            BulkCursor u;
            int c0, yy, xx;
            c0 = bulk_locate<TW>(L, j0, yy, xx);
            cursor_load<TW>(L, u, c0, j0);
            long long job = j0;
            for (; job < j1 && !abort_flag; ++job) {
                const long long t = job - j0;
                const int k = (int)(t % NST);
                if (t >= NST &&
                    !bar_wait_unless(&empty[k], (unsigned)(((t / NST) - 1) & 1), kBulkSpinLimit, abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                while (job >= u.end) cursor_load<TW>(L, u, u.c + 1, job);
                bulk_issue<S>(u, stages + k * 9 * RS, &full[k], &desc[k]);
                if (++u.seg == u.nseg) {
                    u.seg = 0;
                    ++u.y;
                }
            }
            if (abort_flag) {
                // report, then wait (bounded) for copies that may still be landing
                atomicOr(const_cast<unsigned*>(&L.cases[c0]->status), STAT_TIMEOUT);
                for (long long jj = job - 1; jj >= j0 && jj >= job - NST; --jj)
                    bar_wait(&full[(jj - j0) % NST], (unsigned)(((jj - j0) / NST) & 1), kBulkSpinLimit);
            }
        }
        return;
    }

    // consumer warps
    const int lane = tid & 31;
    const long poll_limit = g_consumer_poll_limit;
    ScCase<S> K;
    int cur = -1;
    for (long long job = j0; job < j1; ++job) {
        const long long t = job - j0;
        const int k = (int)(t % NST);
        if (!bar_wait(&full[k], (unsigned)((t / NST) & 1), poll_limit) || abort_flag) {
            abort_flag = 1;
            break;
        }
        const BulkDesc dk = desc[k];
        if (dk.c != cur) {
            K.load(L.cases[dk.c]);
            cur = dk.c;
        }
        const bool forced = (dk.flags & BULK_IB) || K.has_force;
        const S* st = stages + k * 9 * RS + tid + H;
        S* d = K.dst + ((long long)dk.y * K.pitch + dk.x0 + tid);
        const bool unstable = forced ? bulk_tile<S, KIND, true>(K, st, d, dk.x0, dk.y, dk.flags, tid)
                                     : bulk_tile<S, KIND, false>(K, st, d, dk.x0, dk.y, dk.flags, tid);
        if (__any_sync(0xffffffffu, unstable) && lane == 0)
            atomicOr(const_cast<unsigned*>(&K.C->status), STAT_UNSTABLE);
        __syncwarp();
        if (lane == 0) bar_arrive(&empty[k]);   // this warp is done with stage k
    }
}

// ------------------------------------------------------------------------------------------
// Block helpers (fixed-order reductions so results do not depend on timing).
constexpr int kIbThreads = 512;   // threads of the per-body IB CTA
// Warp butterflies, then one warp over the warp results: a fixed combination
// order for any timing, two block barriers instead of one per tree level.
__device__ __forceinline__ double block_max(double v, double* sh) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double u = lane < kIbThreads / 32 ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
        if (lane == 0) sh[kIbThreads / 32] = u;
    }
    __syncthreads();
    return sh[kIbThreads / 32];
}
// Square root of the largest of the threads' non-negative e2, computed once.  The
// maximum runs on the integer pipes (the bit patterns of non-negative doubles order
// as their values), since FP64 arithmetic is scarce on B300.
__device__ __forceinline__ double block_max_sqrt(double e2, double* sh) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    long long v = __double_as_longlong(e2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    long long* shl = reinterpret_cast<long long*>(sh);
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0) shl[w] = v;
    __syncthreads();
    if (w == 0) {
        long long u = lane < kIbThreads / 32 ? shl[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
        if (lane == 0) sh[kIbThreads / 32] = sqrt(__longlong_as_double(u));
    }
    __syncthreads();
    return sh[kIbThreads / 32];
}
// Three FP64 sums in a fixed order: every thread parks its partials in shared memory
// and one warp adds them (lane l takes slots l, l + 32, ...), then a butterfly; few
// FP64 instructions, since FP64 arithmetic is scarce on B300.  sh holds 3 kIbThreads.
// The adding warp's part: lane l sums slots l, l + 32, ... of each array, then a butterfly
// (every lane ends with the totals).
__device__ __forceinline__ void warp_sum3(const double* sh, int lane, double& x, double& y, double& z) {
    x = 0.0; y = 0.0; z = 0.0;
    for (int i = lane; i < kIbThreads; i += 32) {
        x += sh[i];
        y += sh[kIbThreads + i];
        z += sh[2 * kIbThreads + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
        z += __shfl_xor_sync(0xffffffffu, z, o);
    }
}
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    __syncthreads();
    sh[t] = a; sh[kIbThreads + t] = b; sh[2 * kIbThreads + t] = c;
    __syncthreads();
    if (w == 0) {
        double x, y, z;
        warp_sum3(sh, lane, x, y, z);
        __syncwarp();
        if (lane == 0) { sh[0] = x; sh[1] = y; sh[2] = z; }
    }
    __syncthreads();
    a = sh[0]; b = sh[1]; c = sh[2];
}
__device__ __forceinline__ int block_min_i(int v, int* sh) {
    const int t = threadIdx.x;
    __syncthreads();
    sh[t] = v;
    __syncthreads();
    for (int s = kIbThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = min(sh[t], sh[t + s]);
        __syncthreads();
    }
    const int r = sh[0];
    __syncthreads();
    return r;
}
__device__ __forceinline__ int block_max_i(int v, int* sh) {
    const int t = threadIdx.x;
    __syncthreads();
    sh[t] = v;
    __syncthreads();
    for (int s = kIbThreads / 2; s > 0; s >>= 1) {
        if (t < s) sh[t] = max(sh[t], sh[t + s]);
        __syncthreads();
    }
    const int r = sh[0];
    __syncthreads();
    return r;
}

// Block-wide minimum of five ints: warp butterflies, then one warp over the 16 warp
// results (two barriers instead of one per tree level).  sh holds 96 ints.
__device__ __forceinline__ void block_min5(int (&v)[5], int* sh) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 5; ++q) v[q] = min(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) sh[q * 16 + w] = v[q];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            int u = lane < kIbThreads / 32 ? sh[q * 16 + lane] : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u = min(u, __shfl_xor_sync(0xffffffffu, u, o));
            if (lane == 0) sh[80 + q] = u;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 5; ++q) v[q] = sh[80 + q];
}

// Block-wide exclusive scan of two ints (warp scans, then one warp over the warp totals);
// returns the totals.  sh holds 96 ints.
__device__ __forceinline__ void block_exscan2(int& a, int& b, int& tot_a, int& tot_b, int* sh) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ua = __shfl_up_sync(0xffffffffu, ia, o), ub = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += ua;
            ib += ub;
        }
    }
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 31) {
        sh[w] = ia;
        sh[16 + w] = ib;
    }
    __syncthreads();
    if (w == 0) {
        const int xa = lane < kIbThreads / 32 ? sh[lane] : 0, xb = lane < kIbThreads / 32 ? sh[16 + lane] : 0;
        int sa = xa, sb = xb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int ua = __shfl_up_sync(0xffffffffu, sa, o), ub = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += ua;
                sb += ub;
            }
        }
        if (lane < kIbThreads / 32) {
            sh[32 + lane] = sa - xa;
            sh[48 + lane] = sb - xb;
        }
        if (lane == kIbThreads / 32 - 1) {
            sh[64] = sa;
            sh[65] = sb;
        }
    }
    __syncthreads();
    a = sh[32 + w] + ia - a;
    b = sh[48 + w] + ib - b;
    tot_a = sh[64];
    tot_b = sh[65];
}

// Footprint of a body: stencil origins and weights, bounding box, box-local
// node -> slot map and a node -> marker CSR whose lists are sorted by marker
// index (so every spread sums in ascending marker order, like Eq. 8 written out).
// The node map, list fill counters, lists and stencil weights of a footprint rebuild in
// shared memory (a moving body rebuilds it every step): the same slots, list order and
// weights as the global-memory build below, written out once at the end.
constexpr int kFastSmem = 160 * 1024;   // bytes of the IB CTA's dynamic shared memory the fast path may use
constexpr int kFootSmemArea = 6144;   // box nodes
constexpr int kFootSmemEnt = 8192;    // node->marker entries (markers x stencil nodes)
// scratch layout (ints): map, fill, offsets (area + 1, padded to area + 4), entries, origins
// (2 per marker), then 8 weights per marker; kIbThreads markers at most
constexpr int kFootSmemInts = 3 * kFootSmemArea + 4 + kFootSmemEnt + 2 * kIbThreads;
static_assert(kFootSmemInts % 2 == 0, "the weights start 8-byte aligned");
static_assert(kFootSmemInts * 4 + 8 * kIbThreads * 8 <= kFastSmem, "footprint scratch fits the IB CTA's region");
template <class R>
__device__ bool footprint_in_smem(BodyDev& B, int* shi, int* scratch, int bx0, int by0, int bw, int bh) {
    const int tid = threadIdx.x, n = B.n, Sx = B.S, SS = Sx * Sx, ne = n * SS, area = bw * bh;
    int* sMap = scratch;                           // [area] counts, then slot or -1
    int* sFill = sMap + kFootSmemArea;             // [area] fill counters per slot
    int* sOff = sFill + kFootSmemArea;             // [area + 1] list offsets per slot
    int* sEnt = sOff + kFootSmemArea + 4;          // [ne] list entries
    int* sIJ = sEnt + kFootSmemEnt;                // [2n] stencil origins
    R* sW = reinterpret_cast<R*>(scratch + kFootSmemInts);   // [8n] weights
    const R* wts = static_cast<const R*>(B.wts);
    for (int q = tid; q < area; q += kIbThreads) sMap[q] = 0;
    for (int k = tid; k < n; k += kIbThreads) {    // (this thread wrote them: no barrier needed)
        sIJ[2 * k] = B.ij[2 * k];
        sIJ[2 * k + 1] = B.ij[2 * k + 1];
#pragma unroll
        for (int a = 0; a < 8; ++a) sW[k * 8 + a] = wts[k * 8 + a];
    }
    __syncthreads();
    for (int en = tid; en < ne; en += kIbThreads) {
        const int k = en / SS, r = en % SS, b = r / Sx, a = r % Sx;
        atomicAdd(&sMap[(sIJ[2 * k + 1] + b - by0) * bw + (sIJ[2 * k] + a - bx0)], 1);
    }
    __syncthreads();
    // chunked exclusive scans: slot index and list offset (as in the global build)
    const int chunk = (area + kIbThreads - 1) / kIbThreads;
    const int beg = min(area, tid * chunk), end = min(area, beg + chunk);
    int nz = 0, cnt = 0;
    for (int q = beg; q < end; ++q) {
        const int c = sMap[q];
        nz += c > 0;
        cnt += c;
    }
    int slot = nz, off = cnt, tot_nz = 0, tot_cnt = 0;
    block_exscan2(slot, off, tot_nz, tot_cnt, shi);
    for (int q = beg; q < end; ++q) {
        const int c = sMap[q];
        if (c > 0) {
            B.fp_node[slot] = q;
            sOff[slot] = off;
            sFill[slot] = 0;
            sMap[q] = slot;
            ++slot;
            off += c;
        } else {
            sMap[q] = -1;
        }
    }
    const int nfp = tot_nz;
    if (tid == 0) {
        sOff[nfp] = tot_cnt;
        B.bx0 = bx0; B.by0 = by0; B.bw = bw; B.bh = bh; B.nfp = nfp;
    }
    __syncthreads();
    for (int en = tid; en < ne; en += kIbThreads) {
        const int k = en / SS, r = en % SS, b = r / Sx, a = r % Sx;
        const int sl = sMap[(sIJ[2 * k + 1] + b - by0) * bw + (sIJ[2 * k] + a - bx0)];
        B.mslot[en] = sl;
        sEnt[sOff[sl] + atomicAdd(&sFill[sl], 1)] = en;
    }
    __syncthreads();
    R* cw = static_cast<R*>(B.csr_w);
    for (int q = tid; q < nfp; q += kIbThreads) {   // insertion sort of each short list
        const int o0 = sOff[q], o1 = sOff[q + 1];
        for (int i = o0 + 1; i < o1; ++i) {
            const int v = sEnt[i];
            int j = i - 1;
            while (j >= o0 && sEnt[j] > v) {
                sEnt[j + 1] = sEnt[j];
                --j;
            }
            sEnt[j + 1] = v;
        }
        B.csr_off[q] = o0;
        for (int o = o0; o < o1; ++o) {             // D(x - X_k) of each entry, kept with it
            const int en = sEnt[o], k = en / SS, r = en % SS;
            B.csr_ent[o] = en;
            cw[o] = sW[k * 8 + (r % Sx)] * sW[k * 8 + 4 + (r / Sx)];
        }
    }
    if (tid == 0) B.csr_off[nfp] = tot_cnt;
    for (int q = tid; q < area; q += kIbThreads) B.node_map[q] = sMap[q];
    __syncthreads();
    return true;
}

template <class R>
__device__ bool build_footprint(const CaseDev& C, BodyDev& B, int* shi, int* scratch = nullptr) {
    const int tid = threadIdx.x, n = B.n, Sx = B.S, SS = Sx * Sx, kern = B.kernel;
    R* wts = static_cast<R*>(B.wts);
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, err = 0;
    for (int k = tid; k < n; k += kIbThreads) {
        const double X = B.X[k], Y = B.Y[k];
        // range first, in FP64: a diverged body can put markers at coordinates whose
        // conversion to int would overflow (NaN fails these comparisons too)
        if (!(X >= 0.0 && X < (double)C.nx && Y >= 0.0 && Y < (double)C.ny)) {
            err = 1;
            continue;
        }
        const int i0 = (int)floor(X) - (Sx == 4 ? 1 : 0), j0 = (int)floor(Y) - (Sx == 4 ? 1 : 0);
        if (i0 < 0 || j0 < 0 || i0 + Sx > C.nx || j0 + Sx > C.ny) err = 1;
        B.ij[2 * k] = i0;
        B.ij[2 * k + 1] = j0;
        for (int a = 0; a < Sx; ++a) {
            wts[k * 8 + a] = phi<R>(kern, R((double)(i0 + a) - X));
            wts[k * 8 + 4 + a] = phi<R>(kern, R((double)(j0 + a) - Y));
        }
        mnx = min(mnx, i0); mny = min(mny, j0); mxx = max(mxx, i0); mxy = max(mxy, j0);
    }
    int red[5] = {-err, mnx, mny, mxx == INT_MIN ? INT_MAX : -mxx, mxy == INT_MIN ? INT_MAX : -mxy};
    block_min5(red, shi);
    const int e = -red[0];
    const int bx0 = red[1], by0 = red[2];
    if (e) {   // (the box below is meaningless then)
        if (tid == 0) {
            B.nfp = 0;
            B.status |= STAT_MARKER_OUT;
            atomicOr(const_cast<unsigned*>(&C.status), STAT_MARKER_OUT);
        }
        __syncthreads();
        return false;
    }
    const int bx1 = -red[3] + Sx, by1 = -red[4] + Sx;
    const int bw = bx1 - bx0, bh = by1 - by0;
    if (e || (long long)bw * bh > B.box_cap) {
        if (tid == 0) {
            B.nfp = 0;
            B.status |= e ? STAT_MARKER_OUT : STAT_CAPACITY;
            atomicOr(const_cast<unsigned*>(&C.status), e ? STAT_MARKER_OUT : STAT_CAPACITY);
        }
        __syncthreads();
        return false;
    }
    const int area = bw * bh;
    if (scratch && area <= kFootSmemArea && n * SS <= kFootSmemEnt && n <= kIbThreads)
        return footprint_in_smem<R>(B, shi, scratch, bx0, by0, bw, bh);
    for (int q = tid; q < area; q += kIbThreads) B.node_map[q] = 0;
    __syncthreads();
    for (int en = tid; en < n * SS; en += kIbThreads) {
        const int k = en / SS, r = en % SS, b = r / Sx, a = r % Sx;
        const int node = (B.ij[2 * k + 1] + b - by0) * bw + (B.ij[2 * k] + a - bx0);
        atomicAdd(&B.node_map[node], 1);
    }
    __syncthreads();
    // chunked exclusive scans: slot index and CSR offset
    const int chunk = (area + kIbThreads - 1) / kIbThreads;
    const int beg = min(area, tid * chunk), end = min(area, beg + chunk);
    int nz = 0, cnt = 0;
    for (int q = beg; q < end; ++q) {
        const int c = B.node_map[q];
        nz += c > 0;
        cnt += c;
    }
    int slot = nz, off = cnt, tot_nz = 0, tot_cnt = 0;
    block_exscan2(slot, off, tot_nz, tot_cnt, shi);
    for (int q = beg; q < end; ++q) {
        const int c = B.node_map[q];
        if (c > 0) {
            B.fp_node[slot] = q;
            B.csr_off[slot] = off;
            B.node_map[q] = slot;
            ++slot;
            off += c;
        } else {
            B.node_map[q] = -1;
        }
    }
    const int nfp = tot_nz;
    if (tid == 0) {
        B.csr_off[nfp] = tot_cnt;
        B.bx0 = bx0; B.by0 = by0; B.bw = bw; B.bh = bh; B.nfp = nfp;
    }
    for (int q = tid; q < nfp; q += kIbThreads) B.fill[q] = 0;
    __syncthreads();
    for (int en = tid; en < n * SS; en += kIbThreads) {
        const int k = en / SS, r = en % SS, b = r / Sx, a = r % Sx;
        const int node = (B.ij[2 * k + 1] + b - by0) * bw + (B.ij[2 * k] + a - bx0);
        const int sl = B.node_map[node];
        B.mslot[en] = sl;
        B.csr_ent[B.csr_off[sl] + atomicAdd(&B.fill[sl], 1)] = en;
    }
    __syncthreads();
    R* cw = static_cast<R*>(B.csr_w);
    for (int q = tid; q < nfp; q += kIbThreads) {   // insertion sort of each short list
        const int o0 = B.csr_off[q], o1 = B.csr_off[q + 1];
        for (int i = o0 + 1; i < o1; ++i) {
            const int v = B.csr_ent[i];
            int j = i - 1;
            while (j >= o0 && B.csr_ent[j] > v) {
                B.csr_ent[j + 1] = B.csr_ent[j];
                --j;
            }
            B.csr_ent[j + 1] = v;
        }
        for (int o = o0; o < o1; ++o) {             // D(x - X_k) of each entry, kept with it
            const int en = B.csr_ent[o], k = en / SS, r = en % SS;
            cw[o] = wts[k * 8 + (r % Sx)] * wts[k * 8 + 4 + (r / Sx)];
        }
    }
    __syncthreads();
    return true;
}

// Stencil of marker k: footprint slots and weights D(x - X_k) of its SX x SX nodes,
// ordered b-major (ascending j, then i).  Fixed-width loops let every load of a
// marker's stencil be in flight at once.
template <int SX, class R>
__device__ __forceinline__ void marker_stencil(const BodyDev& B, const R* wts, int k, int (&sl)[SX * SX],
                                               R (&D)[SX * SX]) {
#pragma unroll
    for (int r = 0; r < SX * SX; ++r) {
        sl[r] = B.mslot[k * SX * SX + r];
        D[r] = wts[k * 8 + (r % SX)] * wts[k * 8 + 4 + (r / SX)];
    }
}

constexpr int kSpreadChunk = 8;   // CSR entries whose loads are issued together
constexpr int kMdfNodeCap = 2048; // footprint nodes whose MDF iterate fits in shared memory
constexpr int kMdfEntryCap = 4096; // node->marker entries staged in shared memory for MDF
// Dynamic shared memory of ib_kernel: sU (2 per node), sF (2 per marker), sEw (per
// entry), then sEk (per entry, int).
// The fixed-body fast path (ib_fast) and the shared-memory footprint build use up to
// kFastSmem bytes of the same region (kFastSmem is defined with the footprint build).
template <class R> struct IbSmem {
    static constexpr int mdf = (2 * kMdfNodeCap + 2 * 512 + kMdfEntryCap + kMdfNodeCap) * (int)sizeof(R) +
                               (kMdfEntryCap + kMdfNodeCap + 1) * 4;
    static constexpr int bytes = mdf > kFastSmem ? mdf : kFastSmem;
};

// Parts of the per-body IB stage, as bits: set-up (footprint, omega_MDF, DFC lambda_k),
// gather of the post-streaming state at the footprint nodes, marker forces + spread + body
// sums, and marker forces preset (the coupled MDF sets them between a gather and a spread).
enum { IBP_SETUP = 1, IBP_GATHER = 2, IBP_FORCES = 4, IBP_PRESET = 8 };
enum {
    IB_WHOLE = IBP_SETUP | IBP_GATHER | IBP_FORCES,
    IB_SETUP = IBP_SETUP,
    IB_GATHER = IBP_SETUP | IBP_GATHER,
    IB_FORCES = IBP_FORCES,
    IB_SPREAD = IBP_FORCES | IBP_PRESET
};

// Gather of the post-streaming state at the footprint nodes of body B (thread t of nt):
// rho and u (DF, MDF; u twice, the MDF iterate starts from it) or the nine shifted
// populations (DFC) per node into B.fpdata.  A node's values do not depend on which
// thread computes them.
template <class S>
__device__ void ib_gather(const CaseDev& C, const BodyDev& B, int t, int nt) {
    using R = typename Traits<S>::R;
    const int bx0 = B.bx0, by0 = B.by0, bw = B.bw, nfp = B.nfp, scheme = B.scheme;
    R* fp = static_cast<R*>(B.fpdata);
    const S* src = static_cast<const S*>(C.f[(int)(C.step & 1ull)]);
    // GB footprint nodes per thread at a time: their pulls are issued together
    // (interior nodes pull directly; nodes on a lattice edge take the domain conditions)
    constexpr int GB = sizeof(R) == 8 ? 2 : 4;
    const int cnx = C.nx, cny = C.ny, cpitch = C.pitch;
    const long long cplane = C.plane;
    for (int q0 = t; q0 < nfp; q0 += GB * nt) {
        int gx[GB], gy[GB];
        bool live[GB], inner[GB];
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            const int q = q0 + u * nt;
            live[u] = q < nfp;
            const int node = live[u] ? B.fp_node[q] : 0;
            gx[u] = bx0 + node % bw;
            gy[u] = by0 + node / bw;
            inner[u] = live[u] && gx[u] >= 1 && gx[u] <= cnx - 2 && gy[u] >= 1 && gy[u] <= cny - 2;
        }
        R sb[GB][9];
#pragma unroll
        for (int u = 0; u < GB; ++u)
#pragma unroll
            for (int i = 0; i < 9; ++i)
                sb[u][i] = inner[u] ? ld1(src + i * cplane + (long long)(gy[u] - ey(i)) * cpitch + (gx[u] - ex(i)))
                                    : R(0);
#pragma unroll
        for (int u = 0; u < GB; ++u) {
            if (!live[u]) continue;
            if (!inner[u]) post_stream_node<S, R>(C, src, gx[u], gy[u], sb[u]);
            const R* s = sb[u];
            R* o = fp + (size_t)(q0 + u * nt) * 9;
            if (scheme == SCH_DFC) {
#pragma unroll
                for (int i = 0; i < 9; ++i) o[i] = s[i];
            } else {
                R drho = R(0), jx = R(0), jy = R(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    drho += s[i];
                    jx += R(ex(i)) * s[i];
                    jy += R(ey(i)) * s[i];
                }
                const R rho = R(1) + drho;
                o[0] = rho;
                o[1] = jx / rho;
                o[2] = jy / rho;
                o[3] = o[1];
                o[4] = o[2];
            }
        }
    }
}

// Per-body IB stage (Sec. 2.4-2.7) for a stencil width SX (2 hat, 4 Peskin), the parts in
// `part`.  Returns false when nothing more is to be done for the body in this launch (its
// footprint could not be built, or a set-up-only launch).
template <class S, int SX>
__device__ __forceinline__ bool ib_run(const IbLaunch& L, const BodyRef& ref, int* shi, double* shd,
                                       typename Traits<S>::R* sU, typename Traits<S>::R* sF,
                                       typename Traits<S>::R* sEw, int* sEk, typename Traits<S>::R* sQc,
                                       int* sQo, int part = IB_WHOLE) {
    using R = typename Traits<S>::R;
    constexpr int SS = SX * SX;
    const CaseDev& C = *ref.c;
    BodyDev& B = *ref.b;
    const int tid = threadIdx.x;
    const int n = B.n, scheme = B.scheme;
    if ((part & IBP_SETUP) && !B.cache_valid) {
        if (!build_footprint<R>(C, B, shi, reinterpret_cast<int*>(sU))) return false;
        if (tid == 0) B.cache_valid = (B.motion == MOT_FIXED) ? 1 : 0;
    }
    __syncthreads();
    const int bx0 = B.bx0, bw = B.bw, nfp = B.nfp;
    const R* wts = static_cast<const R*>(B.wts);
    R* fp = static_cast<R*>(B.fpdata);
    R* patch = static_cast<R*>(B.patch);
    R* mk = static_cast<R*>(B.mk);
    const R* cw = static_cast<const R*>(B.csr_w);
    const R ds = R(B.ds);

    // MDF relaxation 1/||A||_inf (Sec. 2.5.2): sum_m A_lm = ds sum_x D_l(x) W(x),
    // W(x) = sum_m D_m(x); computed once on the first step.
    if ((part & IBP_SETUP) && scheme == SCH_MDF && !B.st.omega_valid) {
        for (int q = tid; q < nfp; q += kIbThreads) {
            R w = R(0);
            for (int o = B.csr_off[q]; o < B.csr_off[q + 1]; ++o) w += cw[o];
            patch[(size_t)q * 9] = w;
        }
        __syncthreads();
        double best = 0.0;
        for (int k = tid; k < n; k += kIbThreads) {
            int sl[SS];
            R D[SS];
            marker_stencil<SX, R>(B, wts, k, sl, D);
            double row = 0.0;
#pragma unroll
            for (int r = 0; r < SS; ++r) row += (double)D[r] * (double)patch[(size_t)sl[r] * 9];
            best = fmax(best, row * B.ds);
        }
        best = block_max(best, shd);
        if (tid == 0) {
            if (B.st.mdf_omega <= 0.0) B.st.mdf_omega = 1.0 / best;
            B.st.omega_valid = 1;
        }
        __syncthreads();
    }
    if (L.mode == 1) return false;

    // DFC lambda_k of Eq. 17; W_total sums the markers of every DFC body of the case.
    if ((part & IBP_SETUP) && scheme == SCH_DFC && !(B.lam_valid && C.dfc_all_fixed)) {
        for (int q = tid; q < nfp; q += kIbThreads) {
            const int node = B.fp_node[q];
            const int x = bx0 + node % bw, y = B.by0 + node / bw;
            R w = R(0);
            for (int ob = 0; ob < C.nbodies; ++ob) {
                const BodyDev& O = C.bodies[ob];
                if (O.scheme != SCH_DFC) continue;
                if (ob == ref.index) {
                    for (int o = B.csr_off[q]; o < B.csr_off[q + 1]; ++o) w += cw[o];
                } else {
                    for (int k = 0; k < O.n; ++k) {
                        const double dx = (double)x - O.X[k], dy = (double)y - O.Y[k];
                        if (fabs(dx) >= 2.5 || fabs(dy) >= 2.5) continue;
                        w += phi<R>(O.kernel, R(dx)) * phi<R>(O.kernel, R(dy));
                    }
                }
            }
            patch[(size_t)q * 9] = w;
        }
        __syncthreads();
        for (int k = tid; k < n; k += kIbThreads) {
            int sl[SS];
            R D[SS];
            marker_stencil<SX, R>(B, wts, k, sl, D);
            R ws = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) ws += patch[(size_t)sl[r] * 9] * D[r];
            B.lam[k] = 1.0 / (2.0 * 1.0 * B.ds * (double)ws);
        }
        __syncthreads();
        if (tid == 0) B.lam_valid = 1;
    }

    if (part & IBP_GATHER) ib_gather<S>(C, B, tid, kIbThreads);
    __syncthreads();
    if (!(part & IBP_FORCES)) return true;

    // force and torque on the body (Sec. 2.7), accumulated in FP64 by each thread as its
    // markers' forces are final (ascending k per thread), reduced at the end
    double gxs = 0.0, gys = 0.0, ts = 0.0;
    const double bxc = B.st.xc, byc = B.st.yc;
    auto body_force = [&](int k, double gx, double gy) {
        const double rx = B.X[k] - bxc, ry = B.Y[k] - byc;
        gxs += gx;
        gys += gy;
        ts += rx * gy - ry * gx;
    };
    if (part & IBP_PRESET) {
        // marker forces already final (coupled MDF): mk[16k + 0..1] and B.Fx, B.Fy
        for (int k = tid; k < n; k += kIbThreads) body_force(k, -B.Fx[k] * B.ds, -B.Fy[k] * B.ds);
    } else if (scheme == SCH_DF) {
        // Eq. 7 on rho and u_raw, Eq. 11
        for (int k = tid; k < n; k += kIbThreads) {
            int sl[SS];
            R D[SS];
            marker_stencil<SX, R>(B, wts, k, sl, D);
            R rk = R(0), Ux = R(0), Uy = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) {
                const R* g = fp + (size_t)sl[r] * 9;
                rk += g[0] * D[r];
                Ux += g[1] * D[r];
                Uy += g[2] * D[r];
            }
            const R Fx = R(2) * rk * (R(B.Udx[k]) - Ux), Fy = R(2) * rk * (R(B.Udy[k]) - Uy);
            mk[k * 16 + 0] = Fx;
            mk[k * 16 + 1] = Fy;
            B.Fx[k] = (double)Fx;
            B.Fy[k] = (double)Fy;
            body_force(k, -(double)Fx * B.ds, -(double)Fy * B.ds);
        }
    } else if (scheme == SCH_MDF && n <= kIbThreads && nfp <= kMdfNodeCap && B.csr_off[nfp] <= kMdfEntryCap) {
        // Eqs. 12-14 as below, with each thread holding one marker's stencil, density
        // and running force in registers, the iterate u^(n) at the footprint nodes (sU),
        // F^(n) per marker (sF) and the node->marker lists with their weights (sEk, sEw)
        // in shared memory, and each thread's node list bounds and densities in
        // registers: an iteration touches no global memory.
        const R om = R(B.st.mdf_omega);
        const bool own = tid < n;
        int sl[SS];
        R D[SS];
        R rk = R(0), Fxt = R(0), Fyt = R(0);
        double udx = 0.0, udy = 0.0;
        if (own) {
            marker_stencil<SX, R>(B, wts, tid, sl, D);
#pragma unroll
            for (int q = 0; q < SS; ++q) rk += fp[(size_t)sl[q] * 9] * D[q];
            udx = B.Udx[tid];
            udy = B.Udy[tid];
        }
        // staging: each thread loads a batch of independent values before storing any,
        // so one round trip to memory serves the batch
        {
            const R* __restrict__ gfp = fp;
            const int* __restrict__ gent = B.csr_ent;
            const int* __restrict__ goff = B.csr_off;
            const R* __restrict__ gcw = cw;
            constexpr int QB = kMdfNodeCap / kIbThreads;
            R u0[QB], u1[QB], rh[QB];
            int of[QB];
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                const int q = tid + u * kIbThreads;
                const bool live = q < nfp;
                u0[u] = live ? gfp[(size_t)q * 9 + 3] : R(0);
                u1[u] = live ? gfp[(size_t)q * 9 + 4] : R(0);
                rh[u] = live ? gfp[(size_t)q * 9] : R(1);
                of[u] = q <= nfp ? goff[q] : 0;
            }
#pragma unroll
            for (int u = 0; u < QB; ++u) {
                const int q = tid + u * kIbThreads;
                if (q < nfp) {
                    sU[2 * q] = u0[u];
                    sU[2 * q + 1] = u1[u];
                    sQc[q] = om / (R(2) * rh[u]);   // omega / (2 rho(x)), Eq. 14
                }
                if (q <= nfp) sQo[q] = of[u];
            }
            const int ne = goff[nfp];
            constexpr int EB = 8;
            for (int o0 = tid; o0 < ne; o0 += EB * kIbThreads) {
                int ek[EB];
                R ew[EB];
#pragma unroll
                for (int u = 0; u < EB; ++u) {
                    const int o = o0 + u * kIbThreads;
                    ek[u] = o < ne ? gent[o] : 0;
                    ew[u] = o < ne ? gcw[o] : R(0);
                }
#pragma unroll
                for (int u = 0; u < EB; ++u) {
                    const int o = o0 + u * kIbThreads;
                    if (o < ne) {
                        sEk[o] = ek[u] / SS;
                        sEw[o] = ew[u] * ds;
                    }
                }
            }
            if (nfp == QB * kIbThreads && tid == 0) sQo[nfp] = goff[nfp];
        }
        const R rudx = R(udx), rudy = R(udy);
        __syncthreads();
        int applied = 0;
        double rprev = 0.0, r = 0.0;
        bool guard = false, tol_met = false;
        for (int it = 1; it <= B.mdf_nmax; ++it) {
            double e = 0.0;
            R Fx = R(0), Fy = R(0);
            if (own) {
                R Ux = R(0), Uy = R(0);
#pragma unroll
                for (int q = 0; q < SS; ++q) {
                    Ux += sU[2 * sl[q]] * D[q];
                    Uy += sU[2 * sl[q] + 1] * D[q];
                }
                const double dx = udx - (double)Ux, dy = udy - (double)Uy;
                e = dx * dx + dy * dy;            // squared; the root is taken once below
                Fx = R(2) * rk * (rudx - Ux);     // Eq. 13
                Fy = R(2) * rk * (rudy - Uy);
                sF[2 * tid] = Fx;
                sF[2 * tid + 1] = Fy;
            }
            r = block_max_sqrt(e, shd);   // also publishes sF
            if (applied >= B.mdf_nmin && r < B.mdf_tol) { tol_met = true; break; }
            if (it >= 2 && r > 1.5 * rprev) { guard = true; break; }
            for (int q = tid; q < nfp; q += kIbThreads) {
                R sx = R(0), sy = R(0);
                const int o1 = sQo[q + 1];
                for (int o = sQo[q]; o < o1; ++o) {
                    const int k = sEk[o];
                    const R d = sEw[o];   // D(x - X_k) ds
                    sx += sF[2 * k] * d;
                    sy += sF[2 * k + 1] * d;
                }
                sU[2 * q] += sQc[q] * sx;   // Eq. 14 with the node density
                sU[2 * q + 1] += sQc[q] * sy;
            }
            Fxt += om * Fx;
            Fyt += om * Fy;
            __syncthreads();
            rprev = r;
            ++applied;
        }
        if (own) {
            mk[tid * 16 + 0] = Fxt;
            mk[tid * 16 + 1] = Fyt;
            B.Fx[tid] = (double)Fxt;
            B.Fy[tid] = (double)Fyt;
            body_force(tid, -(double)Fxt * B.ds, -(double)Fyt * B.ds);
        }
        if (tid == 0) {
            B.st.mdf_iters = applied;
            B.st.mdf_res = r;
            B.st.mdf_omega_end = B.st.mdf_omega;
            if (guard || (!tol_met && B.mdf_nmax > B.mdf_nmin)) {
                B.status |= STAT_MDF_WARN;
                atomicOr(const_cast<unsigned*>(&C.status), STAT_MDF_WARN);
            }
        }
    } else if (scheme == SCH_MDF) {
        // Eqs. 12-14: at least N_min increments; tolerance and 1.5x guard are
        // tested on U^(n) before increment n; a diverging iterate is not applied.
        // (Bodies with more markers than threads or footprints above kMdfNodeCap.)
        const R om = R(B.st.mdf_omega);
        for (int k = tid; k < n; k += kIbThreads) {
            int sl[SS];
            R D[SS];
            marker_stencil<SX, R>(B, wts, k, sl, D);
            R rk = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) rk += fp[(size_t)sl[r] * 9] * D[r];
            mk[k * 16 + 2] = rk;
            mk[k * 16 + 3] = R(0);
            mk[k * 16 + 4] = R(0);
        }
        __syncthreads();
        int applied = 0;
        double rprev = 0.0, r = 0.0;
        bool guard = false, tol_met = false;
        for (int it = 1; it <= B.mdf_nmax; ++it) {
            double e = 0.0;
            for (int k = tid; k < n; k += kIbThreads) {
                int sl[SS];
                R D[SS];
                marker_stencil<SX, R>(B, wts, k, sl, D);
                R Ux = R(0), Uy = R(0);
#pragma unroll
                for (int q = 0; q < SS; ++q) {
                    const R* g = fp + (size_t)sl[q] * 9;
                    Ux += g[3] * D[q];
                    Uy += g[4] * D[q];
                }
                const double dx = B.Udx[k] - (double)Ux, dy = B.Udy[k] - (double)Uy;
                e = fmax(e, sqrt(dx * dx + dy * dy));
                mk[k * 16 + 5] = R(2) * mk[k * 16 + 2] * (R(B.Udx[k]) - Ux);   // Eq. 13
                mk[k * 16 + 6] = R(2) * mk[k * 16 + 2] * (R(B.Udy[k]) - Uy);
            }
            r = block_max(e, shd);
            if (applied >= B.mdf_nmin && r < B.mdf_tol) { tol_met = true; break; }
            if (it >= 2 && r > 1.5 * rprev) { guard = true; break; }
            for (int q = tid; q < nfp; q += kIbThreads) {
                R sx = R(0), sy = R(0);
                const int o1 = B.csr_off[q + 1];
                for (int o = B.csr_off[q]; o < o1; o += kSpreadChunk) {
                    int kk[kSpreadChunk];
                    R dd[kSpreadChunk];
#pragma unroll
                    for (int u = 0; u < kSpreadChunk; ++u)
                        if (o + u < o1) { kk[u] = B.csr_ent[o + u] / SS; dd[u] = cw[o + u]; }
#pragma unroll
                    for (int u = 0; u < kSpreadChunk; ++u)
                        if (o + u < o1) {
                            sx += mk[kk[u] * 16 + 5] * dd[u] * ds;
                            sy += mk[kk[u] * 16 + 6] * dd[u] * ds;
                        }
                }
                R* g = fp + (size_t)q * 9;
                g[3] += om / (R(2) * g[0]) * sx;   // Eq. 14 with the node density
                g[4] += om / (R(2) * g[0]) * sy;
            }
            for (int k = tid; k < n; k += kIbThreads) {
                mk[k * 16 + 3] += om * mk[k * 16 + 5];
                mk[k * 16 + 4] += om * mk[k * 16 + 6];
            }
            __syncthreads();
            rprev = r;
            ++applied;
        }
        for (int k = tid; k < n; k += kIbThreads) {
            mk[k * 16 + 0] = mk[k * 16 + 3];
            mk[k * 16 + 1] = mk[k * 16 + 4];
            B.Fx[k] = (double)mk[k * 16 + 3];
            B.Fy[k] = (double)mk[k * 16 + 4];
            body_force(k, -(double)mk[k * 16 + 3] * B.ds, -(double)mk[k * 16 + 4] * B.ds);
        }
        if (tid == 0) {
            B.st.mdf_iters = applied;
            B.st.mdf_res = r;
            B.st.mdf_omega_end = B.st.mdf_omega;
            if (guard || (!tol_met && B.mdf_nmax > B.mdf_nmin)) {
                B.status |= STAT_MDF_WARN;
                atomicOr(const_cast<unsigned*>(&C.status), STAT_MDF_WARN);
            }
        }
    } else {
        // DFC, Eqs. 15, 16, 18, 20 on shifted populations: the w_i parts of
        // f*_opp - f*_i cancel, leaving s*_opp - s*_i + 6 w_i e_i.U_d (rho_f = 1).
        for (int k = tid; k < n; k += kIbThreads) {
            int sl[SS];
            R D[SS];
            marker_stencil<SX, R>(B, wts, k, sl, D);
            R st[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) st[i] = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) {
                const R* g = fp + (size_t)sl[r] * 9;
#pragma unroll
                for (int i = 0; i < 9; ++i) st[i] += g[i] * D[r];
            }
            const R lam = R(B.lam[k]);
            const R udx = R(B.Udx[k]), udy = R(B.Udy[k]);
            R fsx = R(0), fsy = R(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R d = lam * (st[opp(i)] - st[i] + R(6) * wgt<R>(i) * (R(ex(i)) * udx + R(ey(i)) * udy));
                mk[k * 16 + 2 + i] = d;
                fsx += R(ex(i)) * d;
                fsy += R(ey(i)) * d;
            }
            mk[k * 16 + 0] = -ds * fsx;
            mk[k * 16 + 1] = -ds * fsy;
            B.Fx[k] = (double)(-ds * fsx);
            B.Fy[k] = (double)(-ds * fsy);
            body_force(k, (double)(-ds * fsx), (double)(-ds * fsy));
        }
    }
    __syncthreads();

    // spread (Eq. 8 / Eq. 19) as a gather over each node's marker list in ascending order
    for (int q = tid; q < nfp; q += kIbThreads) {
        R p[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) p[i] = R(0);
        const int o1 = B.csr_off[q + 1];
        for (int o = B.csr_off[q]; o < o1; o += kSpreadChunk) {
            int kk[kSpreadChunk];
            R dd[kSpreadChunk];
#pragma unroll
            for (int u = 0; u < kSpreadChunk; ++u)
                if (o + u < o1) { kk[u] = B.csr_ent[o + u] / SS; dd[u] = cw[o + u]; }
            if (scheme == SCH_DFC) {
#pragma unroll
                for (int u = 0; u < kSpreadChunk; ++u)
                    if (o + u < o1) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) p[i] += mk[kk[u] * 16 + 2 + i] * dd[u] * ds;
                    }
            } else {
#pragma unroll
                for (int u = 0; u < kSpreadChunk; ++u)
                    if (o + u < o1) {
                        p[0] += mk[kk[u] * 16 + 0] * dd[u] * ds;
                        p[1] += mk[kk[u] * 16 + 1] * dd[u] * ds;
                    }
            }
        }
        // (a DF or MDF patch is read as the force only: p[0], p[1])
        R* o = patch + (size_t)q * 9;
        if (scheme == SCH_DFC) {
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i] = p[i];
        } else {
            o[0] = p[0];
            o[1] = p[1];
        }
    }

    // body force and torque: fixed-order reduction of the per-thread sums
    block_sum3(gxs, gys, ts, shd);
    if (tid == 0) {
        const double Fhx = gxs, Fhy = gys, Th = ts;
        B.st.Fhx = Fhx;
        B.st.Fhy = Fhy;
        B.st.Th = Th;
        const long long h = B.st.hist_n % B.hist_cap;
        B.hist[3 * h + 0] = Fhx;
        B.hist[3 * h + 1] = Fhy;
        B.hist[3 * h + 2] = Th;
        B.st.hist_n = B.st.hist_n + 1;
    }
    return true;
}

__device__ void body_prepare(BodyDev& B, double* sh);
__device__ void body_finish(BodyDev& B);

// Global node index of footprint slot q of body B.
__device__ __forceinline__ int slot_node(const BodyDev& B, int nx, int q) {
    const int node = B.fp_node[q];
    return (B.by0 + node / B.bw) * nx + B.bx0 + node % B.bw;
}

// Marker m of the coupled set -> (body index in C, marker index in that body).
__device__ __forceinline__ void coupled_marker(const CaseDev& C, const int* list, int nb, const int* off, int m,
                                               int& b, int& k) {
    int j = 0;
    while (j + 1 < nb && off[j + 1] <= m) ++j;
    b = list[j];
    k = m - off[j];
}

// Interpolation weights and global nodes of marker k of B (its SX x SX stencil).
template <class R>
__device__ __forceinline__ int marker_nodes(const BodyDev& B, int nx, int k, int (&g)[16], R (&D)[16]) {
    const int SX = B.S, SS = SX * SX;
    const R* wts = static_cast<const R*>(B.wts);
    for (int r = 0; r < SS; ++r) {
        g[r] = slot_node(B, nx, B.mslot[k * SS + r]);
        D[r] = wts[k * 8 + (r % SX)] * wts[k * 8 + 4 + (r / SX)];
    }
    return SS;
}

// Coupled MDF of every MDF body of the case (Sec. 2.5.2, two or more of them), run by
// one CTA after each body's footprint gather.  The bodies' marker forces share one
// fluid update per iteration: S(x) = sum_b spread_b(F_b) (bodies in index order, each
// node summing its markers in ascending order), and, Eq. 12-14 being linear in the
// iterate, a trial with relaxation omega moves every marker velocity to
// U + omega G(k), G(k) = sum_x D(x - X_k) S(x) / (2 rho(x)), so a rejected trial is
// retried with omega / 2 at no extra spreading.  omega_0 = min(0.8, omega_MDF of the
// bodies); a trial whose L_inf residual (FP64, all markers) exceeds 1.2 times the
// current one is rejected and omega halved, ending the iteration at 0.125 omega_0; every
// trial counts towards N_max; at least N_min accepted increments precede a tolerance
// stop; N_min, N_max and tol are the first MDF body's.  Marker scratch mk[16k + ...]:
// 2 rho_k, 3-4 F_total, 5-6 F, 7-8 U, 9-10 G.
template <class S>
__device__ void mdf_coupled(const CaseDev& C, int* shi, double* shd) {
    using R = typename Traits<S>::R;
    const int tid = threadIdx.x, nx = C.nx;
    const long long N = (long long)C.nx * C.ny;
    R* Sx = static_cast<R*>(C.cpl);
    R* Sy = Sx + N;
    R* Q = Sy + N;
    int* list = shi;              // MDF bodies of the case, ascending index
    int* off = shi + kMaxBodies;  // first coupled marker of each (plus the total)
    __syncthreads();
    if (tid == 0) {
        int nb = 0, m = 0;
        for (int b = 0; b < C.nbodies; ++b)
            if (C.bodies[b].scheme == SCH_MDF) {
                list[nb] = b;
                off[nb] = m;
                m += C.bodies[b].n;
                ++nb;
            }
        off[nb] = m;
        shi[2 * kMaxBodies + 1] = nb;
    }
    __syncthreads();
    const int nb = shi[2 * kMaxBodies + 1], M = off[nb];
    bool ok = true;
    double om0 = 0.8;
    for (int j = 0; j < nb; ++j) {
        ok = ok && C.bodies[list[j]].nfp > 0;
        om0 = fmin(om0, C.bodies[list[j]].st.mdf_omega);
    }
    const BodyDev& B0 = C.bodies[list[0]];
    const int nmin = B0.mdf_nmin, nmax = B0.mdf_nmax;
    const double tol = B0.mdf_tol;
    int trials = 0, applied = 0;
    double ra = 0.0, om = om0;
    bool tol_met = false;
    if (ok) {
        // 1 / (2 rho(x)) at every footprint node; rho_k, U^(0) and F per marker
        for (int j = 0; j < nb; ++j) {
            const BodyDev& B = C.bodies[list[j]];
            const R* fp = static_cast<const R*>(B.fpdata);
            for (int q = tid; q < B.nfp; q += kIbThreads) Q[slot_node(B, nx, q)] = R(1) / (R(2) * fp[(size_t)q * 9]);
        }
        double e2 = 0.0;
        for (int m = tid; m < M; m += kIbThreads) {
            int b, k;
            coupled_marker(C, list, nb, off, m, b, k);
            const BodyDev& B = C.bodies[b];
            const R* fp = static_cast<const R*>(B.fpdata);
            R* mk = static_cast<R*>(B.mk) + (size_t)k * 16;
            int g[16];
            R D[16];
            const int SS = marker_nodes<R>(B, nx, k, g, D);
            R rk = R(0), Ux = R(0), Uy = R(0);
            for (int r = 0; r < SS; ++r) {
                const int q = B.mslot[k * SS + r];
                rk += fp[(size_t)q * 9] * D[r];
                Ux += fp[(size_t)q * 9 + 1] * D[r];
                Uy += fp[(size_t)q * 9 + 2] * D[r];
            }
            const double dx = B.Udx[k] - (double)Ux, dy = B.Udy[k] - (double)Uy;
            e2 = fmax(e2, dx * dx + dy * dy);
            mk[2] = rk;
            mk[3] = R(0);
            mk[4] = R(0);
            mk[5] = R(2) * rk * (R(B.Udx[k]) - Ux);   // Eq. 13
            mk[6] = R(2) * rk * (R(B.Udy[k]) - Uy);
            mk[7] = Ux;
            mk[8] = Uy;
        }
        ra = block_max_sqrt(e2, shd);
        bool need_g = true;
        for (;;) {
            if (applied >= nmin && ra < tol) { tol_met = true; break; }
            if (trials >= nmax) break;
            if (need_g) {
                for (int j = 0; j < nb; ++j) {
                    const BodyDev& B = C.bodies[list[j]];
                    for (int q = tid; q < B.nfp; q += kIbThreads) {
                        const int gq = slot_node(B, nx, q);
                        Sx[gq] = R(0);
                        Sy[gq] = R(0);
                    }
                }
                __syncthreads();
                for (int j = 0; j < nb; ++j) {   // bodies in order: S(x) = sum_b spread_b(F_b)
                    const BodyDev& B = C.bodies[list[j]];
                    const int SS = B.S * B.S;
                    const R* cw = static_cast<const R*>(B.csr_w);
                    const R* mkb = static_cast<const R*>(B.mk);
                    const R ds = R(B.ds);
                    for (int q = tid; q < B.nfp; q += kIbThreads) {
                        R sx = R(0), sy = R(0);
                        for (int o = B.csr_off[q]; o < B.csr_off[q + 1]; ++o) {
                            const int k = B.csr_ent[o] / SS;
                            sx += mkb[(size_t)k * 16 + 5] * cw[o] * ds;
                            sy += mkb[(size_t)k * 16 + 6] * cw[o] * ds;
                        }
                        const int gq = slot_node(B, nx, q);
                        Sx[gq] += sx;
                        Sy[gq] += sy;
                    }
                    __syncthreads();
                }
                for (int m = tid; m < M; m += kIbThreads) {
                    int b, k;
                    coupled_marker(C, list, nb, off, m, b, k);
                    const BodyDev& B = C.bodies[b];
                    R* mk = static_cast<R*>(B.mk) + (size_t)k * 16;
                    int g[16];
                    R D[16];
                    const int SS = marker_nodes<R>(B, nx, k, g, D);
                    R Gx = R(0), Gy = R(0);
                    for (int r = 0; r < SS; ++r) {
                        Gx += Sx[g[r]] * Q[g[r]] * D[r];
                        Gy += Sy[g[r]] * Q[g[r]] * D[r];
                    }
                    mk[9] = Gx;
                    mk[10] = Gy;
                }
                need_g = false;
            }
            // trial: every marker velocity at U + omega G
            const R rom = R(om);
            double t2 = 0.0;
            for (int m = tid; m < M; m += kIbThreads) {
                int b, k;
                coupled_marker(C, list, nb, off, m, b, k);
                const BodyDev& B = C.bodies[b];
                const R* mk = static_cast<const R*>(B.mk) + (size_t)k * 16;
                const double dx = B.Udx[k] - (double)(mk[7] + rom * mk[9]);
                const double dy = B.Udy[k] - (double)(mk[8] + rom * mk[10]);
                t2 = fmax(t2, dx * dx + dy * dy);
            }
            const double rt = block_max_sqrt(t2, shd);
            ++trials;
            if (rt > 1.2 * ra) {          // rejected: keep the iterate, halve the relaxation
                om *= 0.5;
                if (om <= 0.125 * om0) break;
                continue;
            }
            for (int m = tid; m < M; m += kIbThreads) {   // accepted
                int b, k;
                coupled_marker(C, list, nb, off, m, b, k);
                const BodyDev& B = C.bodies[b];
                R* mk = static_cast<R*>(B.mk) + (size_t)k * 16;
                const R Ux = mk[7] + rom * mk[9], Uy = mk[8] + rom * mk[10];
                mk[3] += rom * mk[5];
                mk[4] += rom * mk[6];
                mk[7] = Ux;
                mk[8] = Uy;
                mk[5] = R(2) * mk[2] * (R(B.Udx[k]) - Ux);
                mk[6] = R(2) * mk[2] * (R(B.Udy[k]) - Uy);
            }
            ra = rt;
            ++applied;
            need_g = true;
        }
    }
    // final marker forces for the spread, and the diagnostics of every coupled body
    for (int m = tid; m < M; m += kIbThreads) {
        int b, k;
        coupled_marker(C, list, nb, off, m, b, k);
        BodyDev& B = C.bodies[b];
        R* mk = static_cast<R*>(B.mk) + (size_t)k * 16;
        const R fx = ok ? mk[3] : R(0), fy = ok ? mk[4] : R(0);
        mk[0] = fx;
        mk[1] = fy;
        B.Fx[k] = (double)fx;
        B.Fy[k] = (double)fy;
    }
    if (tid == 0)
        for (int j = 0; j < nb; ++j) {
            BodyDev& B = C.bodies[list[j]];
            B.st.mdf_iters = trials;
            B.st.mdf_res = ra;
            B.st.mdf_omega_end = om;
            if (!tol_met && ok) {
                B.status |= STAT_MDF_WARN;
                atomicOr(const_cast<unsigned*>(&C.status), STAT_MDF_WARN);
            }
        }
    __syncthreads();
}

// One CTA per body.  Mode 0 (a step): body motion (body_prepare), the IB stage, then the
// end-of-step body update (body_finish); mode 1: footprint and omega_MDF only.
// ------------------------------------------------------------------------------------------
// IB stage of a fixed DF or DFC body with a cached footprint (the fast path).  The body's
// static data -- each footprint slot's node, each marker's stencil, weights, desired
// velocity and position, the node->marker lists -- is fetched in one batch of independent
// loads, into registers (per marker, per gathered slot) and shared memory (the lists);
// the gathered state goes straight into rank 0's shared memory (distributed shared memory
// of the cluster) and the marker forces stay there, so the stage waits on about four
// global round trips instead of a dozen.  That matters while the sweep beside it keeps
// the memory system saturated.  Every value is computed by the same expressions in the
// same order as in ib_gather / ib_run, so the results are bit for bit those of the
// general path.
__device__ int g_ib_fast_enabled = 1;   // test knob: 0 forces the general path

// Shared-memory layout of the fast path: gathered state (NV R per slot), marker forces
// (NM R per marker), list offsets, marker index and weight per list entry.
template <class R> struct FastLayout {
    int nv, nm, goff, moff, ooff, eoff, woff, bytes;
    __device__ FastLayout(int scheme, int nfp, int n, int ne) {
        nv = scheme == SCH_DFC ? 9 : 3;
        nm = scheme == SCH_DFC ? 9 : 2;
        goff = 0;
        moff = goff + ((nfp * nv * (int)sizeof(R) + 15) & ~15);
        ooff = moff + ((n * nm * (int)sizeof(R) + 15) & ~15);
        eoff = ooff + (((nfp + 1) * 4 + 15) & ~15);
        woff = eoff + ((ne * 4 + 15) & ~15);
        bytes = woff + ne * (int)sizeof(R);
    }
};

// A DF or DFC body whose footprint, stencils and lambda_k are current fits the fast path
// (its shared-memory layout within kFastSmem, at most one marker per thread).
template <class S>
__device__ __forceinline__ bool ib_fast_fits(const BodyDev& B) {
    using R = typename Traits<S>::R;
    if (!g_ib_fast_enabled || B.nfp <= 0 || B.n > kIbThreads) return false;
    if (B.scheme == SCH_DFC) {
        if (!B.lam_valid) return false;
    } else if (B.scheme != SCH_DF) {
        return false;
    }
    const FastLayout<R> F(B.scheme, B.nfp, B.n, B.n * B.S * B.S);
    return F.bytes <= kFastSmem;
}
// ... and a fixed one with its footprint (and lambda_k) cached takes it without a set-up
template <class S>
__device__ __forceinline__ bool ib_fast_ok(const CaseDev& C, const BodyDev& B) {
    return B.motion == MOT_FIXED && B.cache_valid && (B.scheme != SCH_DFC || C.dfc_all_fixed) && ib_fast_fits<S>(B);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
#ifndef IBLBM_EMULATE
    return (unsigned)__cvta_generic_to_shared(p);
#else
    (void)p;
    return 0u;
#endif
}
__device__ __forceinline__ unsigned cluster_map0(unsigned a) {
#ifndef IBLBM_EMULATE
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;" : "=r"(r) : "r"(a));
    return r;
#else
    return a;
#endif
}
__device__ __forceinline__ void st_cluster(unsigned a, float v) {
#ifndef IBLBM_EMULATE
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
#endif
}
__device__ __forceinline__ void st_cluster(unsigned a, double v) {
#ifndef IBLBM_EMULATE
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
#endif
}
__device__ __forceinline__ void cluster_arrive_relaxed() {
#ifndef IBLBM_EMULATE
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
#endif
}
__device__ __forceinline__ void cluster_wait() {
#ifndef IBLBM_EMULATE
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
#endif
}

template <class S, int SX>
__device__ void ib_fast(const IbLaunch& L, const BodyRef& ref, int rank, int G, double* shd, unsigned char* dsm,
                        bool prepare) {
    using R = typename Traits<S>::R;
    constexpr int SS = SX * SX;
    constexpr int GB = sizeof(R) == 8 ? 2 : 4;   // slots per thread whose pulls go out together
    const CaseDev& C = *ref.c;
    BodyDev& B = *ref.b;
    const int tid = threadIdx.x, n = B.n, nfp = B.nfp, ne = n * SS, scheme = B.scheme;
    const FastLayout<R> F(scheme, nfp, n, ne);
    R* sG = reinterpret_cast<R*>(dsm + F.goff);
    R* sM = reinterpret_cast<R*>(dsm + F.moff);
    int* sO = reinterpret_cast<int*>(dsm + F.ooff);
    int* sK = reinterpret_cast<int*>(dsm + F.eoff);
    R* sW = reinterpret_cast<R*>(dsm + F.woff);
    if (G > 1) cluster_arrive_relaxed();   // (every CTA of the cluster has started: DSMEM below)
    // ---- one batch of independent loads: this thread's first slots' nodes, and on rank 0
    // its marker's stencil and weights and its share of the node->marker lists
    const int T = rank * kIbThreads + tid, NT = G * kIbThreads;
    int node0[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u) node0[u] = T + u * NT < nfp ? B.fp_node[T + u * NT] : 0;
    const bool own = rank == 0 && tid < n;
    int sl[SS];
    R wx[4], wy[4];
    // U_d, position and lambda_k of this thread's marker: loaded with the batch when the
    // body motion of the step leaves U_d as it is (a fixed body's usual step), else after it
    const bool ud_static = B.ud_given || B.ud_current;
    double udxk = 0.0, udyk = 0.0, xk = 0.0, yk = 0.0, lamk = 0.0;
    if (own) {
        xk = B.X[tid];
        yk = B.Y[tid];
        if (scheme == SCH_DFC) lamk = B.lam[tid];
        if (ud_static) {
            udxk = B.Udx[tid];
            udyk = B.Udy[tid];
        }
    }
    if (own) {
        const R* wts = static_cast<const R*>(B.wts);
#pragma unroll
        for (int r = 0; r < SS; ++r) sl[r] = B.mslot[tid * SS + r];
#pragma unroll
        for (int a = 0; a < SX; ++a) {
            wx[a] = wts[tid * 8 + a];
            wy[a] = wts[tid * 8 + 4 + a];
        }
    }
    if (rank == 0) {
        const R* cw = static_cast<const R*>(B.csr_w);
        constexpr int EB = 8;   // list entries per thread whose loads go out together
        for (int o0 = tid; o0 <= nfp; o0 += EB * kIbThreads) {
            int v[EB];
#pragma unroll
            for (int u = 0; u < EB; ++u) v[u] = o0 + u * kIbThreads <= nfp ? B.csr_off[o0 + u * kIbThreads] : 0;
#pragma unroll
            for (int u = 0; u < EB; ++u)
                if (o0 + u * kIbThreads <= nfp) sO[o0 + u * kIbThreads] = v[u];
        }
        for (int o0 = tid; o0 < ne; o0 += EB * kIbThreads) {
            int e[EB];
            R w[EB];
#pragma unroll
            for (int u = 0; u < EB; ++u) {
                const int o = o0 + u * kIbThreads;
                e[u] = o < ne ? B.csr_ent[o] : 0;
                w[u] = o < ne ? cw[o] : R(0);
            }
#pragma unroll
            for (int u = 0; u < EB; ++u) {
                const int o = o0 + u * kIbThreads;
                if (o < ne) {
                    sK[o] = e[u] / SS;
                    sW[o] = w[u];
                }
            }
        }
        if (prepare && !L.prepared) body_prepare(B, shd);   // a fixed body: U_d current, or set now
    }
    // ---- gather (every rank): pulls of this thread's slots, rho and u (DF) or the nine
    // shifted populations (DFC) into rank 0's shared memory
    {
        const S* src = static_cast<const S*>(C.f[(int)(C.step & 1ull)]);
        const int bx0 = B.bx0, by0 = B.by0, bw = B.bw;
        const int cnx = C.nx, cny = C.ny, cpitch = C.pitch;
        const long long cplane = C.plane;
        const unsigned g0 = G > 1 ? cluster_map0(smem_u32(sG)) : 0u;
        if (G > 1) cluster_wait();
        for (int q0 = T; q0 < nfp; q0 += GB * NT) {
            int gx[GB], gy[GB];
            bool live[GB], inner[GB];
#pragma unroll
            for (int u = 0; u < GB; ++u) {
                const int q = q0 + u * NT;
                live[u] = q < nfp;
                const int node = !live[u] ? 0 : (q0 == T ? node0[u] : B.fp_node[q]);
                gx[u] = bx0 + node % bw;
                gy[u] = by0 + node / bw;
                inner[u] = live[u] && gx[u] >= 1 && gx[u] <= cnx - 2 && gy[u] >= 1 && gy[u] <= cny - 2;
            }
            R sb[GB][9];
#pragma unroll
            for (int u = 0; u < GB; ++u)
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    sb[u][i] = inner[u] ? ld1(src + i * cplane + (long long)(gy[u] - ey(i)) * cpitch + (gx[u] - ex(i)))
                                        : R(0);
#pragma unroll
            for (int u = 0; u < GB; ++u) {
                if (!live[u]) continue;
                if (!inner[u]) post_stream_node<S, R>(C, src, gx[u], gy[u], sb[u]);
                const R* sv = sb[u];
                const int q = q0 + u * NT;
                R o[9];
                int nvals;
                if (scheme == SCH_DFC) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) o[i] = sv[i];
                    nvals = 9;
                } else {
                    R drho = R(0), jx = R(0), jy = R(0);
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        drho += sv[i];
                        jx += R(ex(i)) * sv[i];
                        jy += R(ey(i)) * sv[i];
                    }
                    const R rho = R(1) + drho;
                    o[0] = rho;
                    o[1] = jx / rho;
                    o[2] = jy / rho;
                    nvals = 3;
                }
                if (G > 1) {
                    for (int j = 0; j < nvals; ++j) st_cluster(g0 + (unsigned)((q * F.nv + j) * (int)sizeof(R)), o[j]);
                } else {
                    for (int j = 0; j < nvals; ++j) sG[q * F.nv + j] = o[j];
                }
            }
        }
    }
    if (G > 1) cluster_sync_all();   // the ranks' gathered values are in rank 0's shared memory
    else __syncthreads();
    if (rank != 0) return;
    // ---- marker forces (one marker per thread), FP64 body sums per thread
    const R ds = R(B.ds);
    double gxs = 0.0, gys = 0.0, ts = 0.0;
    if (own) {
        const int k = tid;
        R D[SS];
#pragma unroll
        for (int r = 0; r < SS; ++r) D[r] = wx[r % SX] * wy[r / SX];
        if (!ud_static) {
            udxk = B.Udx[k];
            udyk = B.Udy[k];
        }
        const double bxc = B.st.xc, byc = B.st.yc;
        const double rx = xk - bxc, ry = yk - byc;
        R* mk = static_cast<R*>(B.mk);
        double fbx, fby;
        if (scheme == SCH_DF) {
            R rk = R(0), Ux = R(0), Uy = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) {
                const R* g = sG + sl[r] * 3;
                rk += g[0] * D[r];
                Ux += g[1] * D[r];
                Uy += g[2] * D[r];
            }
            const R Fx = R(2) * rk * (R(udxk) - Ux), Fy = R(2) * rk * (R(udyk) - Uy);
            sM[2 * k] = Fx;
            sM[2 * k + 1] = Fy;
            mk[k * 16 + 0] = Fx;
            mk[k * 16 + 1] = Fy;
            B.Fx[k] = (double)Fx;
            B.Fy[k] = (double)Fy;
            fbx = -(double)Fx * B.ds;
            fby = -(double)Fy * B.ds;
        } else {
            R st[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) st[i] = R(0);
#pragma unroll
            for (int r = 0; r < SS; ++r) {
                const R* g = sG + sl[r] * 9;
#pragma unroll
                for (int i = 0; i < 9; ++i) st[i] += g[i] * D[r];
            }
            const R lam = R(lamk);
            const R udx = R(udxk), udy = R(udyk);
            R fsx = R(0), fsy = R(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const R d = lam * (st[opp(i)] - st[i] + R(6) * wgt<R>(i) * (R(ex(i)) * udx + R(ey(i)) * udy));
                sM[k * 9 + i] = d;
                mk[k * 16 + 2 + i] = d;
                fsx += R(ex(i)) * d;
                fsy += R(ey(i)) * d;
            }
            mk[k * 16 + 0] = -ds * fsx;
            mk[k * 16 + 1] = -ds * fsy;
            B.Fx[k] = (double)(-ds * fsx);
            B.Fy[k] = (double)(-ds * fsy);
            fbx = (double)(-ds * fsx);
            fby = (double)(-ds * fsy);
        }
        gxs += fbx;
        gys += fby;
        ts += rx * fby - ry * fbx;
    }
    // ---- body force and torque (the fixed-order reduction of block_sum3, by warp 0) beside
    // the spread (Eq. 8 / Eq. 19; each slot's list in ascending marker order, warps 1-15)
    shd[tid] = gxs;
    shd[kIbThreads + tid] = gys;
    shd[2 * kIbThreads + tid] = ts;
    __syncthreads();   // (also publishes the marker forces)
    if (tid < 32) {
        double x, y, z;
        warp_sum3(shd, tid, x, y, z);
        if (tid == 0) {
            B.st.Fhx = x;
            B.st.Fhy = y;
            B.st.Th = z;
            const long long h = B.st.hist_n % B.hist_cap;
            B.hist[3 * h + 0] = x;
            B.hist[3 * h + 1] = y;
            B.hist[3 * h + 2] = z;
            B.st.hist_n = B.st.hist_n + 1;
        }
        return;
    }
    R* patch = static_cast<R*>(B.patch);
    for (int q = tid - 32; q < nfp; q += kIbThreads - 32) {
        R p[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) p[i] = R(0);
        const int o1 = sO[q + 1];
        for (int o = sO[q]; o < o1; ++o) {
            const int k = sK[o];
            const R dd = sW[o];
            if (scheme == SCH_DFC) {
#pragma unroll
                for (int i = 0; i < 9; ++i) p[i] += sM[k * 9 + i] * dd * ds;
            } else {
                p[0] += sM[2 * k] * dd * ds;
                p[1] += sM[2 * k + 1] * dd * ds;
            }
        }
        R* o = patch + (size_t)q * 9;
        if (scheme == SCH_DFC) {
#pragma unroll
            for (int i = 0; i < 9; ++i) o[i] = p[i];
        } else {
            o[0] = p[0];
            o[1] = p[1];
        }
    }
}

template <class S>
__global__ void __launch_bounds__(kIbThreads, 1) ib_kernel(IbLaunch L) {
    if (L.pdl & PDL_TRIGGER) pdl_trigger();
    // L.cluster CTAs per body (a thread-block cluster): rank 0 runs the body's IB stage,
    // the others share the gather of the footprint nodes with it
    const int G = L.cluster > 1 ? L.cluster : 1;
    const int rank = G > 1 ? (int)cluster_rank() : 0;
    const BodyRef ref = L.refs[blockIdx.x / G];
    using R = typename Traits<S>::R;
    static_assert(kIbThreads == 512, "IbSmem sizes sF for 512 markers");
    __shared__ int shi[2 * kIbThreads + 4];
    __shared__ double shd[3 * kIbThreads];
    IBLBM_DYNAMIC_SMEM(dsm);
    R* sU = reinterpret_cast<R*>(dsm);
    R* sF = sU + 2 * kMdfNodeCap;
    R* sEw = sF + 2 * kIbThreads;
    R* sQc = sEw + kMdfEntryCap;
    int* sEk = reinterpret_cast<int*>(sQc + kMdfNodeCap);
    int* sQo = sEk + kMdfEntryCap;
    const CaseDev& C = *ref.c;
    const int SX = ref.b->S;
    if (L.mode == 0 && C.n_mdf >= 2 && ref.b->scheme == SCH_MDF) {
        // coupled MDF: the CTA of the first MDF body steps all of them
        if (ref.index != C.mdf_lead || rank != 0) return;
        if (!L.prepared)
            for (int b = 0; b < C.nbodies; ++b)
                if (C.bodies[b].scheme == SCH_MDF) body_prepare(C.bodies[b], shd);
        for (int b = 0; b < C.nbodies; ++b) {
            if (C.bodies[b].scheme != SCH_MDF) continue;
            const BodyRef rb{ref.c, &C.bodies[b], b, 0};
            if (C.bodies[b].S == 2) ib_run<S, 2>(L, rb, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_GATHER);
            else ib_run<S, 4>(L, rb, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_GATHER);
        }
        mdf_coupled<S>(C, shi, shd);
        for (int b = 0; b < C.nbodies; ++b) {
            if (C.bodies[b].scheme != SCH_MDF) continue;
            const BodyRef rb{ref.c, &C.bodies[b], b, 0};
            if (C.bodies[b].nfp > 0) {
                if (C.bodies[b].S == 2) ib_run<S, 2>(L, rb, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_SPREAD);
                else ib_run<S, 4>(L, rb, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_SPREAD);
            }
            __syncthreads();
            if (threadIdx.x == 0) body_finish(C.bodies[b]);
        }
        return;
    }
    if (L.mode != 0) {   // set-up only: footprint and omega_MDF at the initial markers
        if (rank != 0) return;
        if (SX == 2) ib_run<S, 2>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo);
        else ib_run<S, 4>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo);
        return;
    }
    if (ib_fast_ok<S>(C, *ref.b)) {   // (the same decision on every rank: static fields)
        if (SX == 2) ib_fast<S, 2>(L, ref, rank, G, shd, dsm, true);
        else ib_fast<S, 4>(L, ref, rank, G, shd, dsm, true);
        if (rank == 0) {
            __syncthreads();
            if (threadIdx.x == 0) body_finish(*ref.b);
        }
        return;
    }
    // body motion and set-up (rank 0), gather (every rank), forces, spread, sums and the
    // body update (rank 0).  The ranks' gathered values reach rank 0 through global memory,
    // ordered by the cluster barrier (release / acquire at cluster scope).
    bool ok = true;
    if (rank == 0) {
        if (!L.prepared) body_prepare(*ref.b, shd);
        ok = SX == 2 ? ib_run<S, 2>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_SETUP)
                     : ib_run<S, 4>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_SETUP);
    }
    if (G > 1) cluster_sync_all();
    else __syncthreads();
    // a moving DF or DFC body with its footprint and lambda_k just rebuilt: the rest of the
    // stage on the fast path (the same decision on every rank, from the fields set above;
    // a footprint that could not be built has nfp = 0 and does not fit)
    if (ib_fast_fits<S>(*ref.b)) {
        if (SX == 2) ib_fast<S, 2>(L, ref, rank, G, shd, dsm, false);
        else ib_fast<S, 4>(L, ref, rank, G, shd, dsm, false);
        if (rank == 0) {
            __syncthreads();
            if (threadIdx.x == 0) body_finish(*ref.b);
        }
        return;
    }
    // (a body whose footprint could not be built has nfp = 0: nothing to gather)
    if (ok) ib_gather<S>(C, *ref.b, rank * kIbThreads + (int)threadIdx.x, G * kIbThreads);
    if (G > 1) cluster_sync_all();
    else __syncthreads();
    if (rank != 0) return;
    if (ok) {
        if (SX == 2) ib_run<S, 2>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_FORCES);
        else ib_run<S, 4>(L, ref, shi, shd, sU, sF, sEw, sEk, sQc, sQo, IB_FORCES);
    }
    __syncthreads();
    if (threadIdx.x == 0) body_finish(*ref.b);
}

// ------------------------------------------------------------------------------------------
// Rigid-body motion around the IB stage of a step, run by the body's IB CTA.
// body_prepare (before the IB stage): first half of Eq. 23 with F_total^n = F_h^n + F_g +
// dF_IM^n and the torque-only rotation (FREE), x_c(t) at t = n + 1 (PRESCRIBED), then marker
// positions and U_d = v + omega x (X - X_c); a FIXED body whose desired velocity was set per
// marker keeps it.  body_finish (after it, one thread): second half of Eq. 23 with the force
// just computed and Eq. A3 (FREE), and the body's step counter.
__device__ void body_prepare(BodyDev& B, double* sh) {
    const double PI = 3.14159265358979323846;
    BodyState& S = B.st;
    // a fixed body whose desired velocities are already in place: nothing moves
    if (B.motion == MOT_FIXED && (B.ud_given || B.ud_current)) return;
    const double r2 = B.radius * B.radius;
    const double ms = B.rho_ratio * PI * r2, Is = 0.5 * ms * r2;
    const double dm = (B.rho_ratio - 1.0) * PI * r2;
    __syncthreads();   // sh may still be read by earlier code of the CTA
    if (threadIdx.x == 0) {
        double vx = S.vx, vy = S.vy, om = S.om;
        if (B.motion == MOT_FREE || B.motion == MOT_FREE_TRANSLATION) {
            const double Ftx = S.Fhx + dm * B.gx + S.dFimx, Fty = S.Fhy + dm * B.gy + S.dFimy;
            S.vhx = S.vx + Ftx / (2.0 * ms);
            S.vhy = S.vy + Fty / (2.0 * ms);
            S.omh = B.motion == MOT_FREE ? S.om + S.Th / (2.0 * Is) : 0.0;
            S.xc += S.vhx;
            S.yc += S.vhy;
            S.theta += S.omh;
            vx = S.vhx; vy = S.vhy; om = S.omh;
        } else if (B.motion == MOT_PRESC) {
            const double t = (double)(B.t0 + S.nstep + 1);
            const double w = 2.0 * PI / B.osc_period;
            S.xc = B.xc0 - B.osc_amp * sin(w * t);
            S.vx = -B.osc_amp * w * cos(w * t);
            vx = S.vx; vy = 0.0; om = 0.0;
        }
        sh[0] = S.xc; sh[1] = S.yc; sh[2] = vx; sh[3] = vy; sh[4] = om;
        const bool turns = B.motion == MOT_FREE || B.motion == MOT_FREE_TRANSLATION;
        sh[5] = turns ? cos(S.theta) : 1.0;
        sh[6] = turns ? sin(S.theta) : 0.0;
        if (B.motion != MOT_FIXED) B.cache_valid = 0;
    }
    __syncthreads();
    const double xc = sh[0], yc = sh[1], vx = sh[2], vy = sh[3], om = sh[4], ct = sh[5], st = sh[6];
    for (int k = threadIdx.x; k < B.n; k += blockDim.x) {
        double rx, ry;
        if (B.motion == MOT_FREE || B.motion == MOT_FREE_TRANSLATION) {
            rx = ct * B.r0x[k] - st * B.r0y[k];
            ry = st * B.r0x[k] + ct * B.r0y[k];
            B.X[k] = xc + rx;
            B.Y[k] = yc + ry;
        } else if (B.motion == MOT_PRESC) {
            rx = B.r0x[k];
            ry = B.r0y[k];
            B.X[k] = xc + rx;
            B.Y[k] = B.yc0 + ry;
        } else {
            if (B.ud_given) continue;   // desired velocity set per marker by the caller
            rx = B.X[k] - xc;
            ry = B.Y[k] - yc;
        }
        B.Udx[k] = vx - om * ry;
        B.Udy[k] = vy + om * rx;
    }
    __syncthreads();
    if (threadIdx.x == 0 && B.motion == MOT_FIXED) B.ud_current = 1;
}

__device__ void body_finish(BodyDev& B) {
    const double PI = 3.14159265358979323846;
    BodyState& S = B.st;
    if (B.motion == MOT_FREE || B.motion == MOT_FREE_TRANSLATION) {
        const double r2 = B.radius * B.radius;
        const double ms = B.rho_ratio * PI * r2, Is = 0.5 * ms * r2;
        const double dm = (B.rho_ratio - 1.0) * PI * r2, mf = PI * r2;
        const double vnx = S.vhx + (S.Fhx + dm * B.gx + S.dFimx) / (2.0 * ms);
        const double vny = S.vhy + (S.Fhy + dm * B.gy + S.dFimy) / (2.0 * ms);
        const double omn = B.motion == MOT_FREE ? S.omh + S.Th / (2.0 * Is) : 0.0;
        if (B.internal_mass) {
            S.dFimx = mf * (vnx - S.vx);
            S.dFimy = mf * (vny - S.vy);
        } else {
            S.dFimx = 0.0;
            S.dFimy = 0.0;
        }
        S.vx = vnx; S.vy = vny; S.om = omn;
    }
    S.nstep = S.nstep + 1;
}

// Body motion of the step for every body (one CTA each), when an IB launch must not
// move markers that another body's CTA reads.
__global__ void __launch_bounds__(kThreads) prepare_kernel(BodyRef* refs, int n) {
    __shared__ double sh[8];
    if ((int)blockIdx.x < n) body_prepare(*refs[blockIdx.x].b, sh);
}

// Step counters of every case: the last launch of a step (the sweep reads the
// counter's parity to pick its source buffer).
__global__ void __launch_bounds__(kThreads) counter_kernel(CaseDev** cases, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cases[i]->step += 1ull;
}

template <class S>
__global__ void export_kernel(const CaseDev* __restrict__ Cp, double* out, int shifted) {
    using R = typename Traits<S>::R;
    const CaseDev& C = *Cp;
    const S* src = static_cast<const S*>(C.f[(int)(C.step & 1ull)]);
    const long long N = (long long)C.nx * C.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 9 * N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / N);
        const long long r = q % N;
        const int y = (int)(r / C.nx), x = (int)(r % C.nx);
        const double v = (double)ld1(src + i * C.plane + (long long)y * C.pitch + x);
        out[q] = shifted ? v : v + wgt<double>(i);
    }
}

template <class S>
__global__ void import_kernel(const CaseDev* __restrict__ Cp, const double* in) {
    const CaseDev& C = *Cp;
    S* dst = static_cast<S*>(C.f[(int)(C.step & 1ull)]);
    const long long N = (long long)C.nx * C.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 9 * N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / N);
        const long long r = q % N;
        const int y = (int)(r / C.nx), x = (int)(r % C.nx);
        st1_from_double(dst + i * C.plane + (long long)y * C.pitch + x, in[q] - wgt<double>(i));
    }
}

template <class S>
__global__ void fill_eq_kernel(const CaseDev* __restrict__ Cp, double rho, double ux, double uy) {
    const CaseDev& C = *Cp;
    const long long N = (long long)C.plane;
    const double uu = ux * ux + uy * uy;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 9 * N; q += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(q / N);
        const double v = seq_i<double>(i, rho - 1.0, rho, ux, uy, uu);
        st1_from_double(static_cast<S*>(C.f[0]) + q, v);
        st1_from_double(static_cast<S*>(C.f[1]) + q, v);
    }
}

// Density and Eq. 4 velocity of the last collision at node (x, y), from the stored
// post-collision state: its first moment is rho u + F/2 for the force F of that step.
template <class S>
__device__ __forceinline__ void node_macro(const CaseDev& C, const S* src, int x, int y, double& r, double& u,
                                           double& v) {
    using R = typename Traits<S>::R;
    double drho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double f = (double)ld1(src + i * C.plane + (long long)y * C.pitch + x);
        drho += f;
        jx += ex(i) * f;
        jy += ey(i) * f;
    }
    R s[9];
    for (int i = 0; i < 9; ++i) s[i] = R(0);
    R Fx = R(C.gfx), Fy = R(C.gfy);
    add_ib<R>(C, x, y, s, Fx, Fy);
    r = 1.0 + drho;
    u = (jx - 0.5 * (double)Fx) / r;
    v = (jy - 0.5 * (double)Fy) / r;
}

template <class S>
__global__ void macro_kernel(const CaseDev* __restrict__ Cp, double* rho, double* ux, double* uy) {
    const CaseDev& C = *Cp;
    const S* src = static_cast<const S*>(C.f[(int)(C.step & 1ull)]);
    const long long N = (long long)C.nx * C.ny;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(q / C.nx), x = (int)(q % C.nx);
        node_macro<S>(C, src, x, y, rho[q], ux[q], uy[q]);
    }
}

// ------------------------------------------------------------------------------------------
// Local boundary-fidelity diagnostics of one body (Sec. 2.8; bilinear probe of Sec. 4.2),
// one CTA.  Per marker: the fluid velocity and density interpolated with the body's own
// kernel (Eq. 7) and with the bilinear probe from node_macro, the slip against the
// marker's desired velocity, the normal velocity through the marker polygon (outward
// normal of the chord X_{k+1} - X_{k-1}; radial below three markers) and |F_k|.  Inside
// the body the nodes with |x - X_c| < R - kappa give the residual against the rigid
// velocity v + omega x (x - X_c).  out[0..7] as the C-ABI documents, out[8] = 1 when a
// stencil or probe node lies outside the lattice; pm[5n] (or null) per marker.
constexpr int kDiagThreads = 256;

template <class S>
__global__ void __launch_bounds__(kDiagThreads) diag_kernel(const CaseDev* __restrict__ Cp, int body, double u_ref,
                                                          double kappa, double* __restrict__ out,
                                                          double* __restrict__ pm) {
    __shared__ double red[7][kDiagThreads];
    __shared__ long long cnt_s[kDiagThreads];
    __shared__ int bad_s[kDiagThreads];
    const CaseDev& C = *Cp;
    const BodyDev& B = C.bodies[body];
    const S* src = static_cast<const S*>(C.f[(int)(C.step & 1ull)]);
    const int tid = threadIdx.x, n = B.n, kern = B.kernel, SW = kern == K_HAT ? 2 : 4;
    const double xc = B.st.xc, yc = B.st.yc, ds = B.ds;
    double slip_sum = 0.0, slip_max = 0.0, bl_max = 0.0, net = 0.0, gross = 0.0, fsum = 0.0;
    int bad = 0;
    for (int k = tid; k < n; k += kDiagThreads) {
        const double X = B.X[k], Y = B.Y[k], Udx = B.Udx[k], Udy = B.Udy[k];
        if (!(X >= 0.0 && X < (double)C.nx && Y >= 0.0 && Y < (double)C.ny)) {   // before any int conversion
            bad = 1;
            continue;
        }
        const int b0 = (int)floor(X), c0 = (int)floor(Y);
        const int i0 = b0 - (kern == K_HAT ? 0 : 1), j0 = c0 - (kern == K_HAT ? 0 : 1);
        if (!(X == X) || !(Y == Y) || i0 < 0 || j0 < 0 || i0 + SW > C.nx || j0 + SW > C.ny || b0 < 0 || c0 < 0 ||
            b0 + 2 > C.nx || c0 + 2 > C.ny) {
            bad = 1;
            continue;
        }
        double U = 0.0, V = 0.0, rk = 0.0;
        for (int b = 0; b < SW; ++b) {
            const double py = phi<double>(kern, (double)(j0 + b) - Y);
            for (int a = 0; a < SW; ++a) {
                const double D = phi<double>(kern, (double)(i0 + a) - X) * py;
                double r, u, v;
                node_macro<S>(C, src, i0 + a, j0 + b, r, u, v);
                U += u * D;
                V += v * D;
                rk += r * D;
            }
        }
        const double fx = X - b0, fy = Y - c0;
        double Ub = 0.0, Vb = 0.0, rb = 0.0;
        for (int c = 0; c < 4; ++c) {
            const int a = c & 1, b = c >> 1;
            const double w = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
            double r, u, v;
            node_macro<S>(C, src, b0 + a, c0 + b, r, u, v);
            Ub += u * w;
            Vb += v * w;
            rb += r * w;
        }
        double nxk = 0.0, nyk = 0.0;
        if (n >= 3) {
            const int kp = k + 1 == n ? 0 : k + 1, km = k == 0 ? n - 1 : k - 1;
            const double tx = B.X[kp] - B.X[km], ty = B.Y[kp] - B.Y[km];
            const double t = sqrt(tx * tx + ty * ty);
            if (t > 0.0) {
                nxk = ty / t;
                nyk = -tx / t;
            }
            if (nxk * (X - xc) + nyk * (Y - yc) < 0.0) {
                nxk = -nxk;
                nyk = -nyk;
            }
        } else {
            const double r = sqrt((X - xc) * (X - xc) + (Y - yc) * (Y - yc));
            if (r > 0.0) {
                nxk = (X - xc) / r;
                nyk = (Y - yc) / r;
            }
        }
        const double s = sqrt((U - Udx) * (U - Udx) + (V - Udy) * (V - Udy)) / u_ref;
        const double sb = sqrt((Ub - Udx) * (Ub - Udx) + (Vb - Udy) * (Vb - Udy)) / u_ref;
        const double un = (U - Udx) * nxk + (V - Udy) * nyk;
        const double fm = sqrt(B.Fx[k] * B.Fx[k] + B.Fy[k] * B.Fy[k]);
        slip_sum += s;
        slip_max = fmax(slip_max, s);
        bl_max = fmax(bl_max, sb);
        net += rk * un * ds;
        gross += rk * fabs(un) * ds;
        fsum += fm;
        if (pm) {
            pm[5 * k + 0] = s;
            pm[5 * k + 1] = sb;
            pm[5 * k + 2] = un / u_ref;
            pm[5 * k + 3] = (rb - 1.0) / 3.0;
            pm[5 * k + 4] = fm;
        }
    }
    // interior nodes beyond the buffer; the strict test is taken with single roundings
    // (no fused multiply-add) so that it decides every node as a plain FP64 evaluation does
    double in_sum = 0.0;
    long long cnt = 0;
    const double ri = B.radius - kappa;
    if (ri > 0.0) {
        const double rr = __dmul_rn(ri, ri);
        // clamp to the lattice in FP64 before converting (a diverged body may be anywhere)
        const double fx0 = fmax(0.0, floor(xc - ri)), fx1 = fmin((double)(C.nx - 1), ceil(xc + ri));
        const double fy0 = fmax(0.0, floor(yc - ri)), fy1 = fmin((double)(C.ny - 1), ceil(yc + ri));
        const bool inside = fx1 >= fx0 && fy1 >= fy0;   // false for NaN too
        const int x0 = inside ? (int)fx0 : 0, x1 = inside ? (int)fx1 : -1;
        const int y0 = inside ? (int)fy0 : 0, y1 = inside ? (int)fy1 : -1;
        const int bw = x1 - x0 + 1, bh = y1 - y0 + 1;
        if (bw > 0 && bh > 0) {
            for (long long q = tid; q < (long long)bw * bh; q += kDiagThreads) {
                const int x = x0 + (int)(q % bw), y = y0 + (int)(q / bw);
                const double dx = (double)x - xc, dy = (double)y - yc;
                if (__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) < rr) {
                    double r, u, v;
                    node_macro<S>(C, src, x, y, r, u, v);
                    const double eu = u - (B.st.vx - B.st.om * dy), ev = v - (B.st.vy + B.st.om * dx);
                    in_sum += sqrt(eu * eu + ev * ev);
                    ++cnt;
                }
            }
        }
    }
    red[0][tid] = slip_sum;
    red[1][tid] = slip_max;
    red[2][tid] = bl_max;
    red[3][tid] = net;
    red[4][tid] = gross;
    red[5][tid] = fsum;
    red[6][tid] = in_sum;
    cnt_s[tid] = cnt;
    bad_s[tid] = bad;
    __syncthreads();
    if (tid == 0) {
        double a[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        long long c = 0;
        int anybad = 0;
        for (int t = 0; t < kDiagThreads; ++t) {
            a[0] += red[0][t];
            a[1] = fmax(a[1], red[1][t]);
            a[2] = fmax(a[2], red[2][t]);
            a[3] += red[3][t];
            a[4] += red[4][t];
            a[5] += red[5][t];
            a[6] += red[6][t];
            c += cnt_s[t];
            anybad |= bad_s[t];
        }
        const double norm = u_ref * n * ds;
        out[0] = n > 0 ? a[0] / n : 0.0;
        out[1] = a[1];
        out[2] = a[2];
        out[3] = n > 0 ? a[3] / norm : 0.0;
        out[4] = n > 0 ? a[4] / norm : 0.0;
        out[5] = c > 0 ? a[6] / (double)c / u_ref : 0.0;
        out[6] = (double)c;
        out[7] = a[5];
        out[8] = anybad ? 1.0 : 0.0;
    }
}

cudaError_t launch_diagnostics(const CaseDev* hc, CaseDev* dc, int body, double u_ref, double kappa, double* out,
                               double* pm, cudaStream_t st) {
    switch (hc->storage) {
    case ST_F64: IBLBM_LAUNCH(diag_kernel<double>, 1, kDiagThreads, st, dc, body, u_ref, kappa, out, pm); break;
    case ST_F32: IBLBM_LAUNCH(diag_kernel<float>, 1, kDiagThreads, st, dc, body, u_ref, kappa, out, pm); break;
    default: IBLBM_LAUNCH(diag_kernel<__half>, 1, kDiagThreads, st, dc, body, u_ref, kappa, out, pm); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
static int grid_for(long long work) {
    long long g = (work + 255) / 256;
    if (g > 148 * 32) g = 148 * 32;
    if (g < 1) g = 1;
    return (int)g;
}

template <class S, int KIND>
static cudaError_t sc_launch_k(int variant, const ScLaunch& L, long long jobs, int grid, cudaStream_t st) {
    const int block = L.block > 0 ? L.block : kThreads;
    const bool dep = (L.pdl & PDL_DEPENDENT) != 0;
    if (L.phase == SC_LIST) {
        if (variant == SC_SCALAR) IBLBM_LAUNCH((sc_kernel_list<S, KIND, 1>), grid, block, st, L, jobs);
        else IBLBM_LAUNCH((sc_kernel_list<S, KIND, 2>), grid, block, st, L, jobs);
        return cudaGetLastError();
    }
    if (L.phase == SC_SKIP_IB) {
        if (variant == SC_SCALAR)
            IBLBM_LAUNCH_PDL((sc_kernel_scalar<S, KIND, 1, SC_MODE_SKIP>), grid, block, st, dep, L, jobs);
        else IBLBM_LAUNCH_PDL((sc_kernel_scalar<S, KIND, 2, SC_MODE_SKIP>), grid, block, st, dep, L, jobs);
        return cudaGetLastError();
    }
    if (L.phase == SC_ALL_TAIL) {
        if (variant == SC_SCALAR) IBLBM_LAUNCH((sc_kernel_scalar<S, KIND, 1, SC_MODE_TAIL>), grid, block, st, L, jobs);
        else IBLBM_LAUNCH((sc_kernel_scalar<S, KIND, 2, SC_MODE_TAIL>), grid, block, st, L, jobs);
        return cudaGetLastError();
    }
    if (variant == SC_SCALAR) IBLBM_LAUNCH((sc_kernel_scalar<S, KIND, 1, SC_MODE_PLAIN>), grid, block, st, L, jobs);
    else if (variant == SC_SCALAR2)
        IBLBM_LAUNCH((sc_kernel_scalar<S, KIND, 2, SC_MODE_PLAIN>), grid, block, st, L, jobs);
    else if (variant == SC_BULK) {
        static const cudaError_t attr =
            cudaFuncSetAttribute(reinterpret_cast<const void*>(&sc_kernel_bulk<S, KIND>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, BulkGeom<S>::SMEM);
        if (attr != cudaSuccess) return attr;
        IBLBM_LAUNCH_SMEM((sc_kernel_bulk<S, KIND>), grid, kBulkThreads, BulkGeom<S>::SMEM, st, L, jobs);
    } else IBLBM_LAUNCH((sc_kernel<S, KIND>), grid, kThreads, st, L, jobs);
    return cudaGetLastError();
}

template <class S>
static cudaError_t sc_launch_s(int collision, int variant, const ScLaunch& L, long long jobs, int grid,
                               cudaStream_t st) {
    switch (collision) {
    case COL_BGK: return sc_launch_k<S, COL_BGK>(variant, L, jobs, grid, st);
    case COL_TRT: return sc_launch_k<S, COL_TRT>(variant, L, jobs, grid, st);
    case COL_CM: return sc_launch_k<S, COL_CM>(variant, L, jobs, grid, st);
    case COL_NONE: return sc_launch_k<S, COL_NONE>(variant, L, jobs, grid, st);
    default: return sc_launch_k<S, -1>(variant, L, jobs, grid, st);
    }
}

cudaError_t launch_stream_collide(int storage, int collision, int variant, const ScLaunch& L, long long jobs,
                                  int grid, cudaStream_t st) {
    if (jobs <= 0) return cudaSuccess;
    switch (storage) {
    case ST_F64: return sc_launch_s<double>(collision, variant, L, jobs, grid, st);
    case ST_F32: return sc_launch_s<float>(collision, variant, L, jobs, grid, st);
    default: return sc_launch_s<__half>(collision, variant, L, jobs, grid, st);
    }
}

template <class S, int KIND>
static int sc_occ_k(int variant) {
    int nb = 1;
    if (variant == SC_SCALAR)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sc_kernel_scalar<S, KIND, 1, SC_MODE_PLAIN>, kThreads, 0);
    else if (variant == SC_SCALAR2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sc_kernel_scalar<S, KIND, 2, SC_MODE_PLAIN>, kThreads, 0);
    else if (variant == SC_BULK) {
        const void* fn = reinterpret_cast<const void*>(&sc_kernel_bulk<S, KIND>);
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, BulkGeom<S>::SMEM);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kBulkThreads, BulkGeom<S>::SMEM);
    } else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sc_kernel<S, KIND>, kThreads, 0);
    return nb;
}

template <class S>
static int sc_occ_s(int collision, int variant) {
    switch (collision) {
    case COL_BGK: return sc_occ_k<S, COL_BGK>(variant);
    case COL_TRT: return sc_occ_k<S, COL_TRT>(variant);
    case COL_CM: return sc_occ_k<S, COL_CM>(variant);
    case COL_NONE: return sc_occ_k<S, COL_NONE>(variant);
    default: return sc_occ_k<S, -1>(variant);
    }
}

int sc_blocks_per_sm(int storage, int collision, int variant) {
    int nb = 1;
    switch (storage) {
    case ST_F64: nb = sc_occ_s<double>(collision, variant); break;
    case ST_F32: nb = sc_occ_s<float>(collision, variant); break;
    default: nb = sc_occ_s<__half>(collision, variant); break;
    }
    return nb < 1 ? 1 : nb;
}

int sc_segment(int storage, int variant) {
    const int V = storage == ST_F64 ? 2 : (storage == ST_F32 ? 4 : 8);
    if (variant == SC_BULK)
        return storage == ST_F64 ? BulkGeom<double>::TW : (storage == ST_F32 ? BulkGeom<float>::TW : BulkGeom<__half>::TW);
    const int pair = storage == ST_F16 ? 2 : 1;   // FP16 scalar variants take adjacent node pairs
    return variant == SC_SCALAR ? 32 * pair : (variant == SC_SCALAR2 ? 64 * pair : 32 * V);
}

bool sc_variant_ok(int variant, const void* f0, const void* f1) {
    // bulk copies need 16-byte aligned population buffers
    return variant != SC_BULK || (((uintptr_t)f0 | (uintptr_t)f1) & 15u) == 0;
}

cudaError_t launch_edges(int storage, const EdgeLaunch& L, cudaStream_t st) {
    if (L.nchunks <= 0) return cudaSuccess;
    const int block = L.block > 0 ? L.block : kThreads;
    const bool dep = (L.pdl & PDL_DEPENDENT) != 0;
    switch (storage) {
    case ST_F64: IBLBM_LAUNCH_PDL(edge_kernel<double>, L.nchunks, block, st, dep, L); break;
    case ST_F32: IBLBM_LAUNCH_PDL(edge_kernel<float>, L.nchunks, block, st, dep, L); break;
    default: IBLBM_LAUNCH_PDL(edge_kernel<__half>, L.nchunks, block, st, dep, L); break;
    }
    return cudaGetLastError();
}

long long lattice_edge_nodes(int nx, int ny) { return edge_count(nx, ny); }

template <class S>
static cudaError_t launch_ib_s(const IbLaunch& L, cudaStream_t st) {
    constexpr int smem = IbSmem<typename Traits<S>::R>::bytes;
    static const cudaError_t attr = cudaFuncSetAttribute(reinterpret_cast<const void*>(&ib_kernel<S>),
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
#ifndef IBLBM_EMULATE
    if (L.cluster > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(L.nrefs * L.cluster);
        cfg.blockDim = dim3(kIbThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = L.cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaLaunchKernelEx(&cfg, ib_kernel<S>, L);
        return cudaGetLastError();
    }
#endif
    IBLBM_LAUNCH_SMEM(ib_kernel<S>, L.nrefs, kIbThreads, smem, st, L);
    return cudaGetLastError();
}

template <class S>
static int ib_cluster_size_s(int nrefs, int sm_budget) {
#ifdef IBLBM_EMULATE
    (void)nrefs; (void)sm_budget;
    return 1;
#else
    constexpr int smem = IbSmem<typename Traits<S>::R>::bytes;
    if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&ib_kernel<S>), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    // clusters of 16 CTAs are a non-portable size: allowed explicitly, used when they fit
    if (cudaFuncSetAttribute(reinterpret_cast<const void*>(&ib_kernel<S>),
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
    for (int g = 16; g >= 2; g /= 2) {
        if ((long long)nrefs * g > sm_budget) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(nrefs * g);
        cfg.blockDim = dim3(kIbThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = g;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, ib_kernel<S>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (nc >= nrefs) return g;
    }
    return 1;
#endif
}

int ib_cluster_size(int storage, int nrefs, int sm_budget) {
    if (nrefs <= 0) return 1;
    switch (storage) {
    case ST_F64: return ib_cluster_size_s<double>(nrefs, sm_budget);
    case ST_F32: return ib_cluster_size_s<float>(nrefs, sm_budget);
    default: return ib_cluster_size_s<__half>(nrefs, sm_budget);
    }
}

cudaError_t launch_ib(int storage, const IbLaunch& L, cudaStream_t st) {
    if (L.nrefs <= 0) return cudaSuccess;
    switch (storage) {
    case ST_F64: return launch_ib_s<double>(L, st);
    case ST_F32: return launch_ib_s<float>(L, st);
    default: return launch_ib_s<__half>(L, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_prepare(BodyRef* refs, int nrefs, cudaStream_t st) {
    if (nrefs <= 0) return cudaSuccess;
    IBLBM_LAUNCH(prepare_kernel, nrefs, kThreads, st, refs, nrefs);
    return cudaGetLastError();
}

cudaError_t launch_counters(CaseDev** cases, int ncases, cudaStream_t st) {
    if (ncases <= 0) return cudaSuccess;
    IBLBM_LAUNCH(counter_kernel, (ncases + kThreads - 1) / kThreads, kThreads, st, cases, ncases);
    return cudaGetLastError();
}

cudaError_t launch_export(const CaseDev* hc, CaseDev* dc, double* out, int shifted, cudaStream_t st) {
    const int g = grid_for(9LL * hc->nx * hc->ny);
    switch (hc->storage) {
    case ST_F64: IBLBM_LAUNCH(export_kernel<double>, g, 256, st, dc, out, shifted); break;
    case ST_F32: IBLBM_LAUNCH(export_kernel<float>, g, 256, st, dc, out, shifted); break;
    default: IBLBM_LAUNCH(export_kernel<__half>, g, 256, st, dc, out, shifted); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_import(const CaseDev* hc, CaseDev* dc, const double* in, cudaStream_t st) {
    const int g = grid_for(9LL * hc->nx * hc->ny);
    switch (hc->storage) {
    case ST_F64: IBLBM_LAUNCH(import_kernel<double>, g, 256, st, dc, in); break;
    case ST_F32: IBLBM_LAUNCH(import_kernel<float>, g, 256, st, dc, in); break;
    default: IBLBM_LAUNCH(import_kernel<__half>, g, 256, st, dc, in); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_equilibrium(const CaseDev* hc, CaseDev* dc, double rho, double ux, double uy, cudaStream_t st) {
    const int g = grid_for(9LL * hc->plane);
    switch (hc->storage) {
    case ST_F64: IBLBM_LAUNCH(fill_eq_kernel<double>, g, 256, st, dc, rho, ux, uy); break;
    case ST_F32: IBLBM_LAUNCH(fill_eq_kernel<float>, g, 256, st, dc, rho, ux, uy); break;
    default: IBLBM_LAUNCH(fill_eq_kernel<__half>, g, 256, st, dc, rho, ux, uy); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_macro(const CaseDev* hc, CaseDev* dc, double* rho, double* ux, double* uy, cudaStream_t st) {
    const int g = grid_for((long long)hc->nx * hc->ny);
    switch (hc->storage) {
    case ST_F64: IBLBM_LAUNCH(macro_kernel<double>, g, 256, st, dc, rho, ux, uy); break;
    case ST_F32: IBLBM_LAUNCH(macro_kernel<float>, g, 256, st, dc, rho, ux, uy); break;
    default: IBLBM_LAUNCH(macro_kernel<__half>, g, 256, st, dc, rho, ux, uy); break;
    }
    return cudaGetLastError();
}

cudaError_t set_ib_fast(int enable) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, (const void*)&g_ib_fast_enabled);
    if (e != cudaSuccess) return e;
    const int v = enable ? 1 : 0;
    return cudaMemcpy(p, &v, sizeof(v), cudaMemcpyHostToDevice);
}

cudaError_t set_consumer_poll_limit(long polls) {
    const long v = polls < 0 ? kBulkSpinLimit : polls;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, (const void*)&g_consumer_poll_limit);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(p, &v, sizeof(v), cudaMemcpyHostToDevice);
}

}  // namespace iblbm
