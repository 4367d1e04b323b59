// Launch descriptors shared by the kernels and the host runtime.
#pragma once

#include "iblbm_dev.cuh"

namespace iblbm {

// A body seen from a launch: its case and its slot in that case.
struct BodyRef {
    CaseDev* c;
    BodyDev* b;
    int index;      // body index within its case
    int pad_;
};

// One stream-collide launch over many cases of one storage type.  Work unit:
// one warp handles one row segment of 32*V nodes of one case; job_off[c] is
// the first job of case c (prefix sum, ncases + 1 entries).
// Phases of a scalar-variant launch: every interior node (SC_ALL); every interior
// node outside the IB regions (SC_SKIP_IB, swept while the IB stage runs); the IB
// regions as an explicit segment list (SC_LIST).  The IB region of a body is its
// footprint box's rows, widened in x to multiples of kIbAlign nodes, so that every
// segment of a scalar variant (32, 64 or 128 nodes) lies wholly inside or outside it.
enum { SC_ALL = 0, SC_SKIP_IB = 1, SC_LIST = 2, SC_ALL_TAIL = 3 };
// Compiled forms of the scalar sweep: every node of the first phase; the overlap order's
// SC_SKIP_IB (IB regions left to the tail CTAs); SC_ALL_TAIL, every node plus tail CTAs
// that take the lattice edges and the step end (the last launch of a launch-by-launch step).
enum { SC_MODE_PLAIN = 0, SC_MODE_SKIP = 1, SC_MODE_TAIL = 2 };
constexpr int kIbAlign = 128;
// Programmatic dependent launch: PDL_TRIGGER, the kernel lets the next launch of its
// stream begin as soon as all its CTAs run; PDL_DEPENDENT, the launch may begin before
// the previous one ends and waits for it (griddepcontrol.wait) before it exits.
enum { PDL_TRIGGER = 1, PDL_DEPENDENT = 2 };

// Lattice-edge nodes: chunk k covers edge nodes [first, end) of case c (at most
// L.block of them); launched after the stream-collide launches of the step.
struct EdgeChunk {
    int c, first, end, pad_;
};

struct ScLaunch {
    CaseDev** cases;
    long long* job_off;
    int ncases;
    int block;   // threads per CTA for the scalar variants (0: kThreads)
    const int4* list;   // IB-region segments (x = index into cases, y = row, z = first node)
    int phase;          // SC_ALL, SC_SKIP_IB or SC_LIST
    int pdl;            // PDL_* flags
    // SC_SKIP_IB with tail_ctas > 0: the last tail_ctas CTAs of the grid (dispatched last,
    // onto the SMs the IB stage gives back) sweep no segment outside the IB regions; they
    // wait for the IB stage to end (griddepcontrol.wait), then sweep the nlist listed
    // IB-region segments and -- in the last launch of a step -- the lattice-edge nodes
    // (echunks: 32-node chunks of ecases), one warp per segment or chunk.  The last CTA to
    // finish (done[0] counts finished CTAs and is reset) advances the step counter of every
    // case in count_cases.
    int tail_ctas;
    long long nlist;
    const EdgeChunk* echunks;
    CaseDev** ecases;
    int nechunks;
    int ncount;
    CaseDev** count_cases;
    unsigned* done;
};

struct IbLaunch {
    BodyRef* refs;
    int nrefs;
    int mode;       // 0: body motion + IB stage + end-of-step body update; 1: set-up only
                    // (footprint and omega_MDF at the initial markers)
    int pdl;        // PDL_* flags (PDL_TRIGGER only)
    int prepared;   // 1: body motion of the step already done by launch_prepare (another
                    // body's IB CTA reads these markers: DFC W_total over several bodies)
    int cluster;    // CTAs per body (a thread-block cluster, 1-16; 0 or 1: one CTA); the
                    // others share the body's footprint gather with the first
};

// host-side launchers (kernels.cu)
// Stream-collide variants: SC_VECTOR holds 16-byte vectors (2/4/8 nodes) per
// lane; SC_SCALAR one node per lane; SC_SCALAR2 two nodes per lane (32 apart);
// SC_BULK stages each tile's source rows in shared memory with bulk async copies.
// A job is one row segment of sc_segment(storage, variant) nodes.
enum { SC_VECTOR = 0, SC_SCALAR = 1, SC_SCALAR2 = 2, SC_BULK = 3, SC_VARIANTS = 4 };
cudaError_t launch_stream_collide(int storage, int collision, int variant, const ScLaunch& L, long long jobs,
                                  int grid, cudaStream_t st);
// true when the variant honours ScLaunch.ctr / phase / list (the scalar variants)
inline bool sc_variant_phased(int variant) { return variant == SC_SCALAR || variant == SC_SCALAR2; }
// IB region test shared by the SC_SKIP_IB launch and the host that builds the SC_LIST table.
__host__ __device__ inline bool in_ib_region(int y, int xseg, int bx0, int by0, int bw, int bh) {
    const int ax0 = (bx0 >= 0 ? bx0 / kIbAlign : -((-bx0 + kIbAlign - 1) / kIbAlign)) * kIbAlign;
    const int ax1 = ((bx0 + bw + kIbAlign - 1) / kIbAlign) * kIbAlign;
    return y >= by0 && y < by0 + bh && xseg >= ax0 && xseg < ax1;
}
int sc_segment(int storage, int variant);
bool sc_variant_ok(int variant, const void* f0, const void* f1);   // alignment a variant needs
struct EdgeLaunch {
    CaseDev** cases;
    EdgeChunk* chunks;
    int nchunks;
    int block;   // threads per CTA: the chunk size, a multiple of 32 up to kThreads
    int noib;    // 1: no edge node lies in a body footprint (no IB patch lookup)
    int pdl;     // PDL_DEPENDENT: may start while the previous launch runs, waits for it at the end
    // When set, the edge launch ends the step: its last CTA (done[0] counts finished CTAs and
    // is reset) advances the step counter of every case in count_cases.
    CaseDev** count_cases;
    int ncount;
    int pad_;
    unsigned* done;
};
cudaError_t launch_edges(int storage, const EdgeLaunch& L, cudaStream_t st);
long long lattice_edge_nodes(int nx, int ny);
cudaError_t launch_ib(int storage, const IbLaunch& L, cudaStream_t st);
// CTAs per body for an IB launch over nrefs bodies of this storage type: the largest of
// 16, 8, 4, 2 whose clusters all fit on the GPU at once within sm_budget SMs, else 1
int ib_cluster_size(int storage, int nrefs, int sm_budget);
// body motion of the step (first half of Eq. 23, markers, U_d) for every body, one CTA
// each, before an IB launch with IbLaunch.prepared = 1
cudaError_t launch_prepare(BodyRef* refs, int nrefs, cudaStream_t st);
// advances the step counter of every case (the last launch of a step)
cudaError_t launch_counters(CaseDev** cases, int ncases, cudaStream_t st);
cudaError_t launch_export(const CaseDev* hc, CaseDev* dc, double* out, int shifted, cudaStream_t st);
cudaError_t launch_import(const CaseDev* hc, CaseDev* dc, const double* in, cudaStream_t st);
cudaError_t launch_fill_equilibrium(const CaseDev* hc, CaseDev* dc, double rho, double ux, double uy, cudaStream_t st);
cudaError_t launch_macro(const CaseDev* hc, CaseDev* dc, double* rho, double* ux, double* uy, cudaStream_t st);
// Sec. 2.8 local diagnostics of one body into out[9] (and pm[5n] unless null), one CTA.
cudaError_t launch_diagnostics(const CaseDev* hc, CaseDev* dc, int body, double u_ref, double kappa, double* out,
                               double* pm, cudaStream_t st);
int sc_blocks_per_sm(int storage, int collision, int variant);
// Polls after which the bulk sweep's consumer warps give up waiting for a staged tile
// (negative: the default bound).  Process-wide; for tests of the give-up path.
cudaError_t set_consumer_poll_limit(long polls);
// 0: every IB stage takes the general path (tests compare it with the fixed-body fast path)
cudaError_t set_ib_fast(int enable);

}  // namespace iblbm
