// C ABI of libiblbm.so (declared in include/iblbm.h): context management,
// device memory, CUDA-graph stepping, batched stepping over many lattices,
// checkpoints and exports.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <vector>

#include "iblbm.h"
#include "internal.h"
#include "kernels.cuh"

using namespace iblbm;

// ------------------------------------------------------------------------------------------
static void forget_plans(iblbm_ctx* c);

namespace {

struct AllocHooks {
    iblbm_alloc_fn alloc = nullptr;
    iblbm_free_fn free_fn = nullptr;
    void* user = nullptr;
};
AllocHooks g_hooks;
std::mutex g_mu;

void* dev_alloc(size_t bytes, cudaStream_t st) {
    bytes = std::max<size_t>(256, (bytes + 255) & ~size_t(255));
    if (g_hooks.alloc) return g_hooks.alloc(bytes, st, g_hooks.user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p, cudaStream_t st) {
    if (!p) return;
    if (g_hooks.free_fn) g_hooks.free_fn(p, st, g_hooks.user);
    else cudaFree(p);
}

int status_from_bits(unsigned bits) {
    if (bits & STAT_TIMEOUT) return IBLBM_ERR_TIMEOUT;
    if (bits & STAT_MARKER_OUT) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
    if (bits & STAT_UNSTABLE) return IBLBM_ERR_UNSTABLE;
    if (bits & STAT_CAPACITY) return IBLBM_ERR_CAPACITY;
    if (bits & STAT_MDF_WARN) return IBLBM_WARN_MDF_NOT_CONVERGED;
    return IBLBM_OK;
}

size_t storage_bytes(int st) { return st == ST_F64 ? 8 : (st == ST_F32 ? 4 : 2); }
size_t real_bytes(int st) { return st == ST_F64 ? 8 : 4; }

struct BodyHost {
    int n = 0;
    int kernel = 0, scheme = 0, motion = 0;
    double xc = 0, yc = 0, reach = 0;   // centre and marker reach for overlap checks
    bool moved = false;                 // markers replaced by iblbm_move_body since it was added
};

struct GraphSet {
    cudaGraphExec_t one = nullptr, many = nullptr;
    int many_steps = 0;
    void reset() {
        if (one) cudaGraphExecDestroy(one);
        if (many) cudaGraphExecDestroy(many);
        one = many = nullptr;
    }
};

}  // namespace

struct iblbm_ctx {
    int device = 0;
    cudaStream_t user_stream = nullptr;
    cudaStream_t work = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    iblbm_lattice_desc desc{};
    int collision = 0;
    double tau = 0;
    CaseDev hc{};                 // host copy of the static case fields
    CaseDev* dc = nullptr;        // device case
    BodyDev* dbodies = nullptr;   // device array [kMaxBodies]
    BodyRef* drefs = nullptr;     // device [kMaxBodies]
    CaseDev** dcases = nullptr;   // device [1]
    std::vector<BodyHost> bodies;
    std::vector<std::pair<void*, size_t>> allocs;
    std::vector<BodyDev> hbodies; // host copies of the static body records (device pointers inside)
    size_t bytes = 0;
    long long steps = 0;
    int version = 0;              // bumped when bodies change; batch plans check it
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Timed {
        cudaEvent_t a, b;
        int stage;                // STAGE_*
    };
    std::vector<Timed> ev_pending;
    double sc_ms = 0;             // stream-collide + lattice-edge launches (iblbm_kernel_timing)
    int sc_count = 0;
    double stage_ms[4] = {0, 0, 0, 0};   // per stage (iblbm_stage_timing)
    int stage_n[4] = {0, 0, 0, 0};

    void* alloc(size_t b) {
        void* p = dev_alloc(b, work);
        if (p) {
            allocs.push_back({p, b});
            bytes += b;
        }
        return p;
    }
};

namespace {

int check(cudaError_t e) {
    if (e == cudaSuccess) return IBLBM_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? IBLBM_ERR_OOM : IBLBM_ERR_CUDA;
}

enum { STAGE_IB = 0, STAGE_SWEEP = 1, STAGE_EDGE = 2, STAGE_COUNTER = 3 };

cudaEvent_t pool_event(iblbm_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_timing(iblbm_ctx* c) {
    for (auto& t : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            if (t.stage == STAGE_SWEEP || t.stage == STAGE_EDGE) {
                c->sc_ms += ms;
                c->sc_count += 1;
            }
            c->stage_ms[t.stage] += ms;
            c->stage_n[t.stage] += 1;
        }
        c->ev_pool.push_back(t.a);
        c->ev_pool.push_back(t.b);
    }
    c->ev_pending.clear();
}

// Brackets one launch with timing events when timer is set.
template <class F>
cudaError_t timed_launch(iblbm_ctx* timer, int stage, cudaStream_t st, F&& launch) {
    if (!timer) return launch();
    cudaEvent_t a = pool_event(timer), b = pool_event(timer);
    cudaEventRecord(a, st);
    const cudaError_t e = launch();
    cudaEventRecord(b, st);
    timer->ev_pending.push_back({a, b, stage});
    return e;
}

int sync_status(iblbm_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->work);
    if (e != cudaSuccess) return check(e);
    unsigned bits = 0;
    e = cudaMemcpy(&bits, &c->dc->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return check(e);
    return status_from_bits(bits);
}

void begin_user(iblbm_ctx* c) {
    cudaEventRecord(c->ev_in, c->user_stream);
    cudaStreamWaitEvent(c->work, c->ev_in, 0);
}
void end_user(iblbm_ctx* c) {
    cudaEventRecord(c->ev_out, c->work);
    cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
}

bool valid_bc(const int* bc) {
    for (int s = 0; s < 4; ++s)
        if (bc[s] < 0 || bc[s] > 2) return false;
    return (bc[0] == BC_PER) == (bc[1] == BC_PER) && (bc[2] == BC_PER) == (bc[3] == BC_PER);
}

int stencil_ok(int S, int nx, int ny, double X, double Y) {
    if (!(X >= 0.0 && X < (double)nx && Y >= 0.0 && Y < (double)ny)) return 0;   // before int conversion
    const int i0 = (int)std::floor(X) - (S == 4 ? 1 : 0), j0 = (int)std::floor(Y) - (S == 4 ? 1 : 0);
    return i0 >= 0 && j0 >= 0 && i0 + S <= nx && j0 + S <= ny;
}

int body_index_ok(iblbm_ctx* c, int id) { return c && id >= 0 && id < (int)c->bodies.size(); }

// Bounding-box capacity of a body whose markers lie within `reach` of its centre.
int box_capacity(double reach, int S) {
    const int side = 2 * (int)std::ceil(reach) + S + 4;
    return side * side;
}

size_t rounded(size_t b) { return std::max<size_t>(256, (b + 255) & ~size_t(255)); }

BodyDev fetch_body(iblbm_ctx* c, int id) {
    BodyDev b;
    cudaMemcpy(&b, &c->dbodies[id], sizeof(BodyDev), cudaMemcpyDeviceToHost);
    return b;
}

}  // namespace

// ------------------------------------------------------------------------------------------
extern "C" {

int iblbm_set_allocator(iblbm_alloc_fn alloc, iblbm_free_fn free_fn, void* user) {
    std::lock_guard<std::mutex> lk(g_mu);
    if ((alloc == nullptr) != (free_fn == nullptr)) return IBLBM_ERR_INVALID_ARG;
    g_hooks.alloc = alloc;
    g_hooks.free_fn = free_fn;
    g_hooks.user = user;
    return IBLBM_OK;
}

const char* iblbm_strerror(int status) {
    switch (status) {
    case IBLBM_OK: return "ok";
    case IBLBM_WARN_MDF_NOT_CONVERGED: return "MDF iteration stopped at N_max or by its divergence guard";
    case IBLBM_ERR_INVALID_ARG: return "invalid argument";
    case IBLBM_ERR_OOM: return "out of device memory";
    case IBLBM_ERR_UNSTABLE: return "non-finite or non-positive density";
    case IBLBM_ERR_MARKER_OUT_OF_DOMAIN: return "a marker footprint left the lattice";
    case IBLBM_ERR_BODY_OVERLAP: return "MDF bodies with overlapping footprints";
    case IBLBM_ERR_TIMEOUT: return "timeout";
    case IBLBM_ERR_NOT_ADMITTED: return "request not admitted";
    case IBLBM_ERR_BUSY: return "busy";
    case IBLBM_ERR_CUDA: return "CUDA runtime error";
    case IBLBM_ERR_NOT_FOUND: return "not found";
    case IBLBM_ERR_CAPACITY: return "buffer too small";
    default: return "unknown status";
    }
}

int iblbm_create(const iblbm_lattice_desc* d, int collision, double tau, iblbm_ctx** out) {
    if (!d || !out) return IBLBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->nx < 3 || d->ny < 3 || d->storage < 0 || d->storage > 2 || !valid_bc(d->bc)) return IBLBM_ERR_INVALID_ARG;
    if (collision < 0 || collision > 3 || !(tau > 0.5) || !std::isfinite(tau)) return IBLBM_ERR_INVALID_ARG;
    if (collision == COL_TRT && !(d->trt_lambda > 0.0)) return IBLBM_ERR_INVALID_ARG;
    if (!(d->init_rho > 0.0)) return IBLBM_ERR_INVALID_ARG;
    if (d->wall_closure != 0 && d->wall_closure != 1) return IBLBM_ERR_INVALID_ARG;
    iblbm_ctx* c = new iblbm_ctx();
    cudaGetDevice(&c->device);
    c->desc = *d;
    c->collision = collision;
    c->tau = tau;
    c->user_stream = static_cast<cudaStream_t>(d->cuda_stream);
    if (cudaStreamCreateWithFlags(&c->work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        iblbm_destroy(c);
        return IBLBM_ERR_CUDA;
    }
    CaseDev& h = c->hc;
    h.nx = d->nx;
    h.ny = d->ny;
    h.pitch = ((d->nx + 1 + 31) / 32) * 32;   // room for one padding column, 16-byte rows
    h.storage = d->storage;
    h.plane = (long long)h.pitch * d->ny;
    h.collision = collision;
    for (int s = 0; s < 4; ++s) {
        h.bc[s] = d->bc[s];
        h.ubc[s][0] = d->u_bc[s][0];
        h.ubc[s][1] = d->u_bc[s][1];
    }
    h.wall_bb = 0;
    for (int s = 0; s < 4; ++s)
        if (d->wall_closure == 1 && d->bc[s] == BC_VEL && d->u_bc[s][0] == 0.0 && d->u_bc[s][1] == 0.0)
            h.wall_bb |= 1 << s;
    h.tau = tau;
    h.omega = 1.0 / tau;
    h.s_e = 1.0 / tau;
    h.s_o = collision == COL_TRT ? 1.0 / (0.5 + d->trt_lambda / (tau - 0.5)) : 1.0 / tau;
    h.cm_sq = d->cm_sq;
    h.cm_se = d->cm_se;
    h.gfx = d->force[0];
    h.gfy = d->force[1];
    h.nbodies = 0;
    h.dfc_all_fixed = 1;
    h.step = 0;
    h.status = 0;
    const size_t fbytes = 9 * (size_t)h.plane * storage_bytes(d->storage);
    h.f[0] = c->alloc(fbytes);
    h.f[1] = c->alloc(fbytes);
    c->dc = static_cast<CaseDev*>(c->alloc(sizeof(CaseDev)));
    c->dbodies = static_cast<BodyDev*>(c->alloc(sizeof(BodyDev) * kMaxBodies));
    c->drefs = static_cast<BodyRef*>(c->alloc(sizeof(BodyRef) * kMaxBodies));
    c->dcases = static_cast<CaseDev**>(c->alloc(sizeof(CaseDev*)));
    if (!h.f[0] || !h.f[1] || !c->dc || !c->dbodies || !c->drefs || !c->dcases) {
        iblbm_destroy(c);
        return IBLBM_ERR_OOM;
    }
    h.bodies = c->dbodies;
    cudaMemsetAsync(h.f[0], 0, fbytes, c->work);
    cudaMemsetAsync(h.f[1], 0, fbytes, c->work);
    cudaMemcpyAsync(c->dc, &h, sizeof(CaseDev), cudaMemcpyHostToDevice, c->work);
    cudaMemcpyAsync(c->dcases, &c->dc, sizeof(CaseDev*), cudaMemcpyHostToDevice, c->work);
    launch_fill_equilibrium(&h, c->dc, d->init_rho, d->init_u[0], d->init_u[1], c->work);
    int rc = check(cudaStreamSynchronize(c->work));
    if (rc) {
        iblbm_destroy(c);
        return rc;
    }
    *out = c;
    return IBLBM_OK;
}

void iblbm_destroy(iblbm_ctx* c) {
    if (!c) return;
    forget_plans(c);
    if (c->work) cudaStreamSynchronize(c->work);
    drain_timing(c);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto& a : c->allocs) dev_free(a.first, c->work);
    if (c->work) cudaStreamSynchronize(c->work);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->work) cudaStreamDestroy(c->work);
    cudaGetLastError();
    delete c;
}

int iblbm_add_body(iblbm_ctx* c, const double* xy, int n, double ds, int kernel, int scheme,
                   const iblbm_body_desc* bd, int* body_id) {
    if (!c || !xy || n <= 0 || !(ds > 0.0) || !bd || kernel < 0 || kernel > 1 || scheme < 0 || scheme > 2)
        return IBLBM_ERR_INVALID_ARG;
    if ((int)c->bodies.size() >= kMaxBodies) return IBLBM_ERR_INVALID_ARG;
    if (bd->motion < 0 || bd->motion > 3 || !(bd->radius > 0.0) || !(bd->rho_ratio > 0.0)) return IBLBM_ERR_INVALID_ARG;
    if (bd->motion == MOT_PRESC && !(bd->osc_period > 0.0)) return IBLBM_ERR_INVALID_ARG;
    if (scheme == SCH_MDF && (bd->mdf_nmin < 0 || bd->mdf_nmax < 1 || bd->mdf_nmin > bd->mdf_nmax)) return IBLBM_ERR_INVALID_ARG;
    const int S = kernel == K_HAT ? 2 : 4;
    double reach = 0.0;
    for (int k = 0; k < n; ++k) {
        if (!stencil_ok(S, c->hc.nx, c->hc.ny, xy[2 * k], xy[2 * k + 1])) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
        reach = std::max(reach, std::hypot(xy[2 * k] - bd->xc, xy[2 * k + 1] - bd->yc));
    }
    const size_t rb = real_bytes(c->hc.storage);
    const int box_cap = box_capacity(reach, S);
    const int nent = n * S * S;
    const int hist_cap = bd->history_cap > 0 ? bd->history_cap : 65536;
    BodyDev B;
    std::memset(&B, 0, sizeof(B));
    B.n = n; B.kernel = kernel; B.scheme = scheme; B.motion = bd->motion;
    B.internal_mass = bd->internal_mass ? 1 : 0;
    B.mdf_nmin = bd->mdf_nmin; B.mdf_nmax = bd->mdf_nmax; B.S = S;
    B.ds = ds; B.radius = bd->radius; B.rho_ratio = bd->rho_ratio; B.gx = bd->gx; B.gy = bd->gy;
    B.mdf_tol = bd->mdf_tol; B.osc_amp = bd->osc_amp; B.osc_period = bd->osc_period > 0 ? bd->osc_period : 1.0;
    B.xc0 = bd->xc; B.yc0 = bd->yc; B.t0 = c->steps;
    B.st.xc = bd->xc; B.st.yc = bd->yc;
    B.st.mdf_omega = bd->mdf_omega;
    B.st.omega_valid = 0;
    B.box_cap = box_cap; B.nent = nent; B.hist_cap = hist_cap;
    B.X = (double*)c->alloc(8 * n); B.Y = (double*)c->alloc(8 * n);
    B.r0x = (double*)c->alloc(8 * n); B.r0y = (double*)c->alloc(8 * n);
    B.Udx = (double*)c->alloc(8 * n); B.Udy = (double*)c->alloc(8 * n);
    B.Fx = (double*)c->alloc(8 * n); B.Fy = (double*)c->alloc(8 * n);
    B.lam = (double*)c->alloc(8 * n);
    B.node_map = (int*)c->alloc(4 * (size_t)box_cap);
    B.fp_node = (int*)c->alloc(4 * (size_t)nent);
    B.csr_off = (int*)c->alloc(4 * (size_t)(nent + 1));
    B.csr_ent = (int*)c->alloc(4 * (size_t)nent);
    B.fill = (int*)c->alloc(4 * (size_t)nent);
    B.csr_w = c->alloc(rb * (size_t)nent);
    B.mslot = (int*)c->alloc(4 * (size_t)nent);
    B.ij = (int*)c->alloc(8 * (size_t)n);
    B.wts = c->alloc(rb * 8 * (size_t)n);
    B.fpdata = c->alloc(rb * 9 * (size_t)nent);
    B.patch = c->alloc(rb * 9 * (size_t)nent);
    B.mk = c->alloc(rb * 16 * (size_t)n);
    B.hist = (double*)c->alloc(24 * (size_t)hist_cap);
    if (!B.X || !B.Y || !B.r0x || !B.r0y || !B.Udx || !B.Udy || !B.Fx || !B.Fy || !B.lam || !B.node_map ||
        !B.fp_node || !B.csr_off || !B.csr_ent || !B.fill || !B.csr_w || !B.mslot || !B.ij || !B.wts || !B.fpdata || !B.patch || !B.mk ||
        !B.hist)
        return IBLBM_ERR_OOM;
    std::vector<double> X(n), Y(n), rx(n), ry(n);
    for (int k = 0; k < n; ++k) {
        X[k] = xy[2 * k];
        Y[k] = xy[2 * k + 1];
        rx[k] = X[k] - bd->xc;
        ry[k] = Y[k] - bd->yc;
    }
    cudaStream_t w = c->work;
    cudaMemcpyAsync(B.X, X.data(), 8 * n, cudaMemcpyHostToDevice, w);
    cudaMemcpyAsync(B.Y, Y.data(), 8 * n, cudaMemcpyHostToDevice, w);
    cudaMemcpyAsync(B.r0x, rx.data(), 8 * n, cudaMemcpyHostToDevice, w);
    cudaMemcpyAsync(B.r0y, ry.data(), 8 * n, cudaMemcpyHostToDevice, w);
    cudaMemsetAsync(B.Udx, 0, 8 * n, w);
    cudaMemsetAsync(B.Udy, 0, 8 * n, w);
    cudaMemsetAsync(B.Fx, 0, 8 * n, w);
    cudaMemsetAsync(B.Fy, 0, 8 * n, w);
    cudaMemsetAsync(B.lam, 0, 8 * n, w);
    cudaMemsetAsync(B.hist, 0, 24 * (size_t)hist_cap, w);
    const int id = (int)c->bodies.size();
    if (scheme == SCH_MDF) {
        // two or more MDF bodies iterate coupled (Sec. 2.5.2) over a lattice-wide scratch
        if (c->hc.n_mdf == 0) c->hc.mdf_lead = id;
        c->hc.n_mdf += 1;
        if (c->hc.n_mdf == 2 && !c->hc.cpl) {
            c->hc.cpl = c->alloc(3 * (size_t)c->hc.nx * c->hc.ny * rb);
            if (!c->hc.cpl) return IBLBM_ERR_OOM;
        }
        cudaMemcpyAsync(&c->dc->n_mdf, &c->hc.n_mdf, sizeof(int), cudaMemcpyHostToDevice, w);
        cudaMemcpyAsync(&c->dc->mdf_lead, &c->hc.mdf_lead, sizeof(int), cudaMemcpyHostToDevice, w);
        cudaMemcpyAsync(&c->dc->cpl, &c->hc.cpl, sizeof(void*), cudaMemcpyHostToDevice, w);
    }
    cudaMemcpyAsync(&c->dbodies[id], &B, sizeof(BodyDev), cudaMemcpyHostToDevice, w);
    BodyRef ref{c->dc, &c->dbodies[id], id, 0};
    cudaMemcpyAsync(&c->drefs[id], &ref, sizeof(BodyRef), cudaMemcpyHostToDevice, w);
    BodyHost bh;
    bh.n = n; bh.kernel = kernel; bh.scheme = scheme; bh.motion = bd->motion;
    bh.xc = bd->xc; bh.yc = bd->yc; bh.reach = reach;
    c->bodies.push_back(bh);
    c->hbodies.push_back(B);
    c->hc.nbodies = (int)c->bodies.size();
    int all_fixed = 1;
    for (auto& o : c->bodies)
        if (o.scheme == SCH_DFC && o.motion != MOT_FIXED) all_fixed = 0;
    c->hc.dfc_all_fixed = all_fixed;
    cudaMemcpyAsync(&c->dc->nbodies, &c->hc.nbodies, sizeof(int), cudaMemcpyHostToDevice, w);
    cudaMemcpyAsync(&c->dc->dfc_all_fixed, &c->hc.dfc_all_fixed, sizeof(int), cudaMemcpyHostToDevice, w);
    // every DFC body re-derives lambda_k now that W_total may include new markers
    for (int b = 0; b < id; ++b) {
        int zero = 0;
        cudaMemcpyAsync(&c->dbodies[b].lam_valid, &zero, sizeof(int), cudaMemcpyHostToDevice, w);
    }
    // MDF relaxation from the markers as given (Sec. 2.5.2: computed once at initialisation)
    if (scheme == SCH_MDF) {
        IbLaunch setup{c->drefs + id, 1, 1, 0, 0};
        int rc = check(launch_ib(c->hc.storage, setup, w));
        if (rc) return rc;
    }
    c->version++;
    if (body_id) *body_id = id;
    return check(cudaStreamSynchronize(w));
}

int iblbm_step(iblbm_ctx* c, int nsteps) {
    if (!c || nsteps < 0) return IBLBM_ERR_INVALID_ARG;
    return iblbm_internal_step_batch(&c, 1, nsteps, 1);   // a batch of one: same plan, graphs and kernels
}

int iblbm_sync(iblbm_ctx* c) {
    if (!c) return IBLBM_ERR_INVALID_ARG;
    return sync_status(c);
}

long long iblbm_steps_done(const iblbm_ctx* c) { return c ? c->steps : -1; }

size_t iblbm_device_bytes(const iblbm_ctx* c) { return c ? c->bytes : 0; }

int iblbm_body_forces(iblbm_ctx* c, int id, double out[3]) {
    if (!body_index_ok(c, id) || !out) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    out[0] = b.st.Fhx; out[1] = b.st.Fhy; out[2] = b.st.Th;
    return rc;
}

int iblbm_body_state(iblbm_ctx* c, int id, double out[6]) {
    if (!body_index_ok(c, id) || !out) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    out[0] = b.st.xc; out[1] = b.st.yc; out[2] = b.st.vx; out[3] = b.st.vy; out[4] = b.st.om; out[5] = b.st.theta;
    return rc;
}

int iblbm_force_history(iblbm_ctx* c, int id, double* out, int cap, int* n) {
    if (!body_index_ok(c, id) || (!out && cap > 0) || cap < 0 || !n) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    const long long have = std::min<long long>(b.st.hist_n, b.hist_cap);
    const long long m = std::min<long long>(have, cap);
    std::vector<double> ring(3 * (size_t)b.hist_cap);
    if (m > 0) cudaMemcpy(ring.data(), b.hist, 24 * (size_t)b.hist_cap, cudaMemcpyDeviceToHost);
    for (long long j = 0; j < m; ++j) {
        const long long step = b.st.hist_n - m + j;
        const long long slot = step % b.hist_cap;
        std::memcpy(out + 3 * j, ring.data() + 3 * slot, 24);
    }
    *n = (int)m;
    return rc;
}

int iblbm_move_body(iblbm_ctx* c, int id, const double* xy, const double uvw[3]) {
    if (!body_index_ok(c, id)) return IBLBM_ERR_INVALID_ARG;
    if (c->bodies[id].motion != MOT_FIXED) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    const int n = b.n;
    if (xy) {
        for (int k = 0; k < n; ++k)
            if (!stencil_ok(b.S, c->hc.nx, c->hc.ny, xy[2 * k], xy[2 * k + 1])) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
        std::vector<double> X(n), Y(n);
        for (int k = 0; k < n; ++k) { X[k] = xy[2 * k]; Y[k] = xy[2 * k + 1]; }
        cudaMemcpy(b.X, X.data(), 8 * n, cudaMemcpyHostToDevice);
        cudaMemcpy(b.Y, Y.data(), 8 * n, cudaMemcpyHostToDevice);
        b.cache_valid = 0;
        b.lam_valid = 0;
        c->bodies[id].moved = true;
        c->version += 1;   // batch plans decide launch order from body positions: rebuild them
    }
    if (uvw) {
        b.st.vx = uvw[0];
        b.st.vy = uvw[1];
        b.st.om = uvw[2];
        b.ud_given = 0;
    }
    b.ud_current = 0;   // U_d recomputed from the new state
    cudaMemcpy(&c->dbodies[id], &b, sizeof(BodyDev), cudaMemcpyHostToDevice);
    if (xy)
        for (int o = 0; o < (int)c->bodies.size(); ++o) {
            int zero = 0;
            cudaMemcpy(&c->dbodies[o].lam_valid, &zero, sizeof(int), cudaMemcpyHostToDevice);
        }
    return check(cudaGetLastError());
}

int iblbm_set_marker_velocity(iblbm_ctx* c, int id, const double* ud) {
    if (!body_index_ok(c, id)) return IBLBM_ERR_INVALID_ARG;
    if (c->bodies[id].motion != MOT_FIXED) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    const int n = b.n;
    if (ud) {
        std::vector<double> U(n), V(n);
        for (int k = 0; k < n; ++k) {
            U[k] = ud[2 * k];
            V[k] = ud[2 * k + 1];
            if (!(std::fabs(U[k]) < 1.0) || !(std::fabs(V[k]) < 1.0)) return IBLBM_ERR_INVALID_ARG;
        }
        cudaMemcpy(b.Udx, U.data(), 8 * (size_t)n, cudaMemcpyHostToDevice);
        cudaMemcpy(b.Udy, V.data(), 8 * (size_t)n, cudaMemcpyHostToDevice);
    }
    const int flag = ud ? 1 : 0, zero = 0;
    cudaMemcpy(&c->dbodies[id].ud_given, &flag, sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(&c->dbodies[id].ud_current, &zero, sizeof(int), cudaMemcpyHostToDevice);
    return check(cudaGetLastError());
}

int iblbm_marker_data(iblbm_ctx* c, int id, double* out) {
    if (!body_index_ok(c, id) || !out) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    const int n = b.n;
    std::vector<double> col(n);
    double* src[7] = {b.X, b.Y, b.Udx, b.Udy, b.Fx, b.Fy, b.lam};
    for (int j = 0; j < 7; ++j) {
        cudaMemcpy(col.data(), src[j], 8 * n, cudaMemcpyDeviceToHost);
        for (int k = 0; k < n; ++k) out[7 * k + j] = (j == 6 && b.scheme != SCH_DFC) ? 0.0 : col[k];
    }
    return check(cudaGetLastError()) ? IBLBM_ERR_CUDA : rc;
}

int iblbm_local_diagnostics(iblbm_ctx* c, int id, double u_ref, double kappa, double out[8], double* per_marker) {
    if (!body_index_ok(c, id) || !out || !(u_ref > 0.0) || !(kappa >= 0.0) || !(u_ref < 1e300) || !(kappa < 1e300))
        return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    const int n = fetch_body(c, id).n;
    const size_t words = 9 + (per_marker ? 5 * (size_t)n : 0);
    double* d = static_cast<double*>(dev_alloc(8 * words, c->work));
    if (!d) return IBLBM_ERR_OOM;
    std::vector<double> h(words);
    int e = check(launch_diagnostics(&c->hc, c->dc, id, u_ref, kappa, d, per_marker ? d + 9 : nullptr, c->work));
    if (!e) e = check(cudaMemcpyAsync(h.data(), d, 8 * words, cudaMemcpyDeviceToHost, c->work));
    if (!e) e = check(cudaStreamSynchronize(c->work));
    dev_free(d, c->work);
    if (e) return e;
    if (h[8] != 0.0) return IBLBM_ERR_MARKER_OUT_OF_DOMAIN;
    std::memcpy(out, h.data(), 8 * sizeof(double));
    if (per_marker) std::memcpy(per_marker, h.data() + 9, 5 * (size_t)n * sizeof(double));
    return rc;
}

int iblbm_marker_stencils(iblbm_ctx* c, int id, int* ij) {
    if (!body_index_ok(c, id) || !ij) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    cudaMemcpy(ij, b.ij, 8 * (size_t)b.n, cudaMemcpyDeviceToHost);
    return check(cudaGetLastError()) ? IBLBM_ERR_CUDA : rc;
}

int iblbm_mdf_info(iblbm_ctx* c, int id, int* iters, double* res, double* omega) {
    if (!body_index_ok(c, id)) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    if (iters) *iters = b.st.mdf_iters;
    if (res) *res = b.st.mdf_res;
    if (omega) *omega = b.st.mdf_omega;
    return rc;
}

int iblbm_mdf_relaxation(iblbm_ctx* c, int id, double* omega_end) {
    if (!body_index_ok(c, id) || !omega_end) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    BodyDev b = fetch_body(c, id);
    *omega_end = b.st.mdf_omega_end;
    return rc;
}

int iblbm_get_populations(iblbm_ctx* c, double* f, int shifted) {
    if (!c || !f) return IBLBM_ERR_INVALID_ARG;
    const size_t N = 9 * (size_t)c->hc.nx * c->hc.ny;
    double* d = static_cast<double*>(dev_alloc(N * 8, c->work));
    if (!d) return IBLBM_ERR_OOM;
    int rc = check(launch_export(&c->hc, c->dc, d, shifted ? 1 : 0, c->work));
    if (!rc) rc = check(cudaMemcpyAsync(f, d, N * 8, cudaMemcpyDeviceToHost, c->work));
    if (!rc) rc = check(cudaStreamSynchronize(c->work));
    dev_free(d, c->work);
    return rc;
}

int iblbm_set_populations(iblbm_ctx* c, const double* f) {
    if (!c || !f) return IBLBM_ERR_INVALID_ARG;
    const size_t N = 9 * (size_t)c->hc.nx * c->hc.ny;
    cudaStreamSynchronize(c->work);
    double* d = static_cast<double*>(dev_alloc(N * 8, c->work));
    if (!d) return IBLBM_ERR_OOM;
    int rc = check(cudaMemcpyAsync(d, f, N * 8, cudaMemcpyHostToDevice, c->work));
    if (!rc) rc = check(launch_import(&c->hc, c->dc, d, c->work));
    if (!rc) rc = check(cudaStreamSynchronize(c->work));
    dev_free(d, c->work);
    return rc;
}

int iblbm_get_macro(iblbm_ctx* c, double* rho, double* ux, double* uy) {
    if (!c || !rho || !ux || !uy) return IBLBM_ERR_INVALID_ARG;
    const size_t N = (size_t)c->hc.nx * c->hc.ny;
    double* d = static_cast<double*>(dev_alloc(3 * N * 8, c->work));
    if (!d) return IBLBM_ERR_OOM;
    int rc = check(launch_macro(&c->hc, c->dc, d, d + N, d + 2 * N, c->work));
    if (!rc) rc = check(cudaMemcpyAsync(rho, d, N * 8, cudaMemcpyDeviceToHost, c->work));
    if (!rc) rc = check(cudaMemcpyAsync(ux, d + N, N * 8, cudaMemcpyDeviceToHost, c->work));
    if (!rc) rc = check(cudaMemcpyAsync(uy, d + 2 * N, N * 8, cudaMemcpyDeviceToHost, c->work));
    if (!rc) rc = check(cudaStreamSynchronize(c->work));
    dev_free(d, c->work);
    return rc;
}

// Checkpoint layout: header, the current population buffer (raw storage), then
// per body: BodyState and the marker arrays X, Y, Udx, Udy, Fx, Fy, lam and the
// force-history ring.
struct SnapHeader {
    unsigned magic;
    int nx, ny, storage, nbodies, pad;
    long long steps;
    unsigned long long dev_step;
};

int iblbm_snapshot(iblbm_ctx* c, void* host, size_t cap, size_t* n) {
    if (!c || !n) return IBLBM_ERR_INVALID_ARG;
    int rc = sync_status(c);
    if (rc < 0) return rc;
    const size_t fb = 9 * (size_t)c->hc.plane * storage_bytes(c->hc.storage);
    size_t total = sizeof(SnapHeader) + fb;
    std::vector<BodyDev> bs;
    for (int b = 0; b < (int)c->bodies.size(); ++b) {
        bs.push_back(fetch_body(c, b));
        total += sizeof(BodyState) + 7 * 8 * (size_t)bs.back().n + 24 * (size_t)bs.back().hist_cap;
    }
    *n = total;
    if (!host) return IBLBM_OK;
    if (cap < total) return IBLBM_ERR_CAPACITY;
    CaseDev dcase;
    cudaMemcpy(&dcase, c->dc, sizeof(CaseDev), cudaMemcpyDeviceToHost);
    char* p = static_cast<char*>(host);
    SnapHeader h{0x49424c4du, c->hc.nx, c->hc.ny, c->hc.storage, (int)c->bodies.size(), 0, c->steps, dcase.step};
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    cudaMemcpy(p, c->hc.f[(int)(dcase.step & 1ull)], fb, cudaMemcpyDeviceToHost);
    p += fb;
    for (auto& b : bs) {
        std::memcpy(p, &b.st, sizeof(BodyState));
        p += sizeof(BodyState);
        double* arr[7] = {b.X, b.Y, b.Udx, b.Udy, b.Fx, b.Fy, b.lam};
        for (int j = 0; j < 7; ++j) {
            cudaMemcpy(p, arr[j], 8 * (size_t)b.n, cudaMemcpyDeviceToHost);
            p += 8 * (size_t)b.n;
        }
        cudaMemcpy(p, b.hist, 24 * (size_t)b.hist_cap, cudaMemcpyDeviceToHost);
        p += 24 * (size_t)b.hist_cap;
    }
    return check(cudaGetLastError()) ? IBLBM_ERR_CUDA : rc;
}

int iblbm_restore(iblbm_ctx* c, const void* host, size_t n) {
    if (!c || !host || n < sizeof(SnapHeader)) return IBLBM_ERR_INVALID_ARG;
    SnapHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != 0x49424c4du || h.nx != c->hc.nx || h.ny != c->hc.ny || h.storage != c->hc.storage ||
        h.nbodies != (int)c->bodies.size())
        return IBLBM_ERR_INVALID_ARG;
    // every copy goes on the context's own stream and the call waits for that stream
    // only: restoring one lattice does not wait for work queued on other lattices
    cudaStream_t w = c->work;
    cudaStreamSynchronize(w);
    const size_t fb = 9 * (size_t)c->hc.plane * storage_bytes(c->hc.storage);
    const char* p = static_cast<const char*>(host) + sizeof(h);
    size_t need = sizeof(h) + fb;
    std::vector<BodyDev> bs;
    for (int b = 0; b < h.nbodies; ++b) {
        bs.emplace_back();
        cudaMemcpyAsync(&bs.back(), &c->dbodies[b], sizeof(BodyDev), cudaMemcpyDeviceToHost, w);
        cudaStreamSynchronize(w);
        need += sizeof(BodyState) + 7 * 8 * (size_t)bs.back().n + 24 * (size_t)bs.back().hist_cap;
    }
    if (n < need) return IBLBM_ERR_INVALID_ARG;
    cudaMemcpyAsync(c->hc.f[(int)(h.dev_step & 1ull)], p, fb, cudaMemcpyHostToDevice, w);
    p += fb;
    cudaMemcpyAsync(&c->dc->step, &h.dev_step, sizeof(unsigned long long), cudaMemcpyHostToDevice, w);
    const unsigned zero = 0;
    cudaMemcpyAsync(&c->dc->status, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, w);
    for (int b = 0; b < h.nbodies; ++b) {
        BodyDev& B = bs[b];
        std::memcpy(&B.st, p, sizeof(BodyState));
        p += sizeof(BodyState);
        double* arr[7] = {B.X, B.Y, B.Udx, B.Udy, B.Fx, B.Fy, B.lam};
        for (int j = 0; j < 7; ++j) {
            cudaMemcpyAsync(arr[j], p, 8 * (size_t)B.n, cudaMemcpyHostToDevice, w);
            p += 8 * (size_t)B.n;
        }
        cudaMemcpyAsync(B.hist, p, 24 * (size_t)B.hist_cap, cudaMemcpyHostToDevice, w);
        p += 24 * (size_t)B.hist_cap;
        B.cache_valid = 0;
        B.lam_valid = 0;
        B.ud_current = 0;
        B.status = 0;
        B.t0 = h.steps - B.st.nstep;   // step at which the body joined the checkpointed run
        cudaMemcpyAsync(&c->dbodies[b], &B, sizeof(BodyDev), cudaMemcpyHostToDevice, w);
    }
    c->steps = h.steps;
    for (int b = 0; b < h.nbodies; ++b) c->hbodies[b].t0 = bs[b].t0;
    c->version += 1;   // footprints are rebuilt: batch plans must build them before overlapping
    return check(cudaStreamSynchronize(w));
}

int iblbm_set_timing(iblbm_ctx* c, int enable) {
    if (!c) return IBLBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->work);
    drain_timing(c);
    c->timing = enable != 0;
    c->sc_ms = 0;
    c->sc_count = 0;
    for (int k = 0; k < 4; ++k) {
        c->stage_ms[k] = 0;
        c->stage_n[k] = 0;
    }
    return IBLBM_OK;
}

int iblbm_stage_timing(iblbm_ctx* c, double ms[4], int launches[4]) {
    if (!c) return IBLBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->work);
    drain_timing(c);
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = c->stage_ms[k];
        if (launches) launches[k] = c->stage_n[k];
        c->stage_ms[k] = 0;
        c->stage_n[k] = 0;
    }
    return IBLBM_OK;
}

int iblbm_kernel_timing(iblbm_ctx* c, double* ms, int* launches) {
    if (!c) return IBLBM_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->work);
    drain_timing(c);
    if (ms) *ms = c->sc_ms;
    if (launches) *launches = c->sc_count;
    c->sc_ms = 0;
    c->sc_count = 0;
    return IBLBM_OK;
}

}  // extern "C"

// Device bytes a lattice plus one body of n markers will hold (mirrors the
// allocations of iblbm_create and iblbm_add_body); used for admission.
size_t iblbm_internal_estimate_bytes(const iblbm_lattice_desc* d, int n, double reach, int kernel, int hist_cap) {
    const size_t pitch = ((size_t)(d->nx + 1 + 31) / 32) * 32;
    const size_t plane = pitch * (size_t)d->ny;
    size_t b = 2 * rounded(9 * plane * storage_bytes(d->storage));
    b += rounded(sizeof(CaseDev)) + rounded(sizeof(BodyDev) * kMaxBodies) + rounded(sizeof(BodyRef) * kMaxBodies) +
         rounded(sizeof(CaseDev*)) + rounded(2 * sizeof(long long));
    if (n > 0) {
        const int S = kernel == K_HAT ? 2 : 4;
        const size_t nent = (size_t)n * S * S, rb = real_bytes(d->storage);
        const size_t hc = hist_cap > 0 ? (size_t)hist_cap : 65536;
        b += 9 * rounded(8 * (size_t)n) + rounded(4 * (size_t)box_capacity(reach, S)) + 4 * rounded(4 * nent) +
             rounded(4 * (nent + 1)) + rounded(8 * (size_t)n) + rounded(rb * 8 * n) + 2 * rounded(rb * 9 * nent) +
             rounded(rb * nent) + rounded(rb * 16 * n) + rounded(24 * hc);
    }
    return b;
}

// ------------------------------------------------------------------------------------------
// Batched stepping: one launch per kernel per storage type per step over a
// case/tile table spanning every lattice of the batch.
namespace {

// Stream-collide group: lattices sharing storage type and collision operator
// (one specialised kernel launch); IB group: bodies of lattices sharing a storage type.
struct BatchGroup {
    int storage = 0;
    int collision = 0;
    int ncases = 0;
    CaseDev** dcases = nullptr;
    long long jobs[SC_VARIANTS] = {};          // per kernel variant (segment widths differ)
    int grid[SC_VARIANTS] = {};
    int block[SC_VARIANTS] = {};               // scalar variants: threads per CTA (0: default)
    long long* djob[SC_VARIANTS] = {};
    bool ok[SC_VARIANTS] = {};                 // variant usable for every lattice of the group
    int size_class = 0;                        // 1: the group sweeps >= kLargeGroupNodes nodes
    int grid_overlap[SC_VARIANTS] = {};        // grid while the IB stage holds some SMs
    int per_sm[SC_VARIANTS] = {};              // resident CTAs per SM at the group's block size
};

// Stream-collide variant per (storage, collision, size class), process-wide so
// that a lattice runs the same kernel alone, in any batch of its class and in the
// server.  Small groups (< kLargeGroupNodes nodes) are latency-bound and tuned
// apart from bandwidth-bound large ones.  -1: not chosen yet; the first plan that
// needs it times every variant in place and keeps the fastest (the kernel
// rewrites only its destination buffer from an unchanged source, so repeating it
// has no effect on the state).
constexpr long long kLargeGroupNodes = 1LL << 20;
int g_variant[3][5][2] = {{{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
                          {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}},
                          {{-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}, {-1, -1}}};
double g_variant_ms[3][5][2][SC_VARIANTS];
static_assert(SC_VARIANTS == IBLBM_KERNEL_VARIANTS, "public variant count must match the kernels");
struct IbGroup {
    int storage = 0;
    BodyRef* drefs = nullptr;
    int nrefs = 0;
    int cluster = 1;                           // CTAs per body (ib_cluster_size)
};
// Lattice-edge nodes of all lattices of one storage type (one launch per step).
struct EdgeGroup {
    int storage = 0;
    CaseDev** dcases = nullptr;
    EdgeChunk* dchunks = nullptr;
    int nchunks = 0;
    int block = 0;                             // edge nodes per chunk = threads per CTA
};

// IB-region segments of the lattices of one stream-collide group, swept after the IB
// stage while the rest of each lattice is swept during it (same specialised kernel as
// the group, so a node's arithmetic does not depend on the order of the launches).
struct ListGroup {
    int storage = 0;
    int collision = 0;
    int group = 0;                             // index into BatchPlan::groups
    CaseDev** dcases = nullptr;                // the group's lattices (list indices into it)
    // per scalar variant (its segment width): the segments, their count and the grid
    int4* dlist[SC_VARIANTS] = {};
    long long n[SC_VARIANTS] = {};
    int grid[SC_VARIANTS] = {};
};

struct BatchPlan {
    std::vector<iblbm_ctx*> ctxs;
    std::vector<int> versions;
    std::vector<BatchGroup> groups;
    std::vector<IbGroup> ib_groups;
    std::vector<EdgeGroup> edge_groups;
    BodyRef* drefs_all = nullptr;
    CaseDev** dcases_all = nullptr;
    int nrefs_all = 0;
    std::vector<void*> mem;
    GraphSet graphs;
    cudaStream_t st = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> joins;
    // Lattice-edge launch overlapped with the IB stage on a side stream, when no body
    // can reach a lattice edge (the edge nodes then need no IB patch).
    bool edges_early = false;
    // Every body fixed with a valid footprint, and few enough bodies: the IB stage runs
    // alongside the sweep of everything outside the IB regions, on SMs the sweep's grid
    // leaves free; the IB-region segments are swept after it (list_groups).
    bool overlap_ok = false;
    std::vector<ListGroup> list_groups;
    // A lattice with several DFC bodies, one of them moving: W_total of Eq. 17 reads every
    // DFC body's markers, so all bodies move in a launch of their own before the IB stage.
    bool prepare_first = false;
    unsigned* ddone = nullptr;                 // finished-CTA count of the step-ending launch
    // One storage type: the last sweep launch of a step takes the lattice edges (32-node
    // chunks) and the end of the step in its tail CTAs; in the overlap order each group's
    // sweep also takes its IB-region segments after the IB stage.  A step is then the IB
    // launch and one launch per group.
    bool fused_tail = false;
    int sms = 148;
    EdgeChunk* dechunks32 = nullptr;
    int nechunks32 = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_edges = nullptr;
    ~BatchPlan() {
        graphs.reset();
        for (auto p : mem) dev_free(p, st);
        for (auto e : joins) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_edges) cudaEventDestroy(ev_edges);
        if (side) cudaStreamDestroy(side);
    }
};

std::map<std::vector<iblbm_ctx*>, BatchPlan*> g_plans;

void* plan_alloc(BatchPlan* P, size_t b) {
    void* p = dev_alloc(b, P->st);
    if (p) P->mem.push_back(p);
    return p;
}

cudaError_t launch_edge_groups(BatchPlan* P, cudaStream_t st, iblbm_ctx* timer, int noib, bool ends_step = false) {
    for (auto& g : P->edge_groups) {
        EdgeLaunch el{g.dcases, g.dchunks, g.nchunks, g.block, noib, 0, nullptr, 0, 0, nullptr};
        if (ends_step) {   // (one edge group): begins beside the launch before it, ends the step
            el.pdl = PDL_DEPENDENT;
            el.count_cases = P->dcases_all;
            el.ncount = (int)P->ctxs.size();
            el.done = P->ddone;
        }
        const cudaError_t e = timed_launch(timer, STAGE_EDGE, st, [&] { return launch_edges(g.storage, el, st); });
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int chosen_variant(const BatchGroup& g) {
    const int chosen = g_variant[g.storage][g.collision][g.size_class];
    int v = chosen < 0 ? SC_SCALAR : chosen;
    return g.ok[v] ? v : SC_SCALAR;
}

// One IB-LBM step of every lattice of the plan.  With every body fixed (overlap): the IB
// stage (body motion, interface coupling, body update; one CTA per body) lets the sweeps
// of the lattices outside their IB regions start at once (programmatic dependent
// launch) and run beside it, then the IB-region segments are swept with the spread
// forces; otherwise the IB stage precedes whole-lattice sweeps.  Lattice-edge nodes run
// on a side stream during the IB stage when no body can reach them, else after the
// sweeps; the step counters advance last.
cudaError_t launch_batch_step(BatchPlan* P, cudaStream_t st, iblbm_ctx* timer) {
    cudaError_t e = cudaSuccess;
    // (not with the vector variant, whose launch also writes side nodes that the edge
    // launch must overwrite afterwards)
    bool early = P->edges_early && !timer;
    bool overlap = P->overlap_ok && !timer;
    for (auto& g : P->groups) {
        const int v = chosen_variant(g);
        if (v == SC_VECTOR) early = false;
        if (!sc_variant_phased(v)) overlap = false;
    }
    // the sweep beside the IB stage needs every free SM slot at once: the edge launch
    // then follows the sweeps instead of running beside them
    if (overlap) early = false;
    if (early) {
        cudaEventRecord(P->ev_fork, st);
        cudaStreamWaitEvent(P->side, P->ev_fork, 0);
        if ((e = launch_edge_groups(P, P->side, nullptr, 1)) != cudaSuccess) return e;
        cudaEventRecord(P->ev_edges, P->side);
    }
    if (P->prepare_first && P->nrefs_all > 0)
        if ((e = timed_launch(timer, STAGE_IB, st, [&] { return launch_prepare(P->drefs_all, P->nrefs_all, st); })) !=
            cudaSuccess)
            return e;
    for (size_t k = 0; k < P->ib_groups.size(); ++k) {
        const auto& g = P->ib_groups[k];
        const bool last = k + 1 == P->ib_groups.size();
        IbLaunch il{g.drefs, g.nrefs, 0, (overlap && last) ? (int)PDL_TRIGGER : 0, P->prepare_first ? 1 : 0,
                    g.cluster};
        if ((e = timed_launch(timer, STAGE_IB, st, [&] { return launch_ib(g.storage, il, st); })) != cudaSuccess)
            return e;
    }
    const bool dependent = overlap && !P->ib_groups.empty();
    const bool fused = dependent && P->fused_tail;
    // launch-by-launch order: the last sweep launch takes the lattice edges and ends the step
    // when its variant has the tail form and the edges did not run beside the IB stage (with
    // nothing else for its tail, the plain form and the counter launch measured faster)
    const bool serial_tail = !overlap && !early && !timer && P->fused_tail && !P->groups.empty() &&
                             sc_variant_phased(chosen_variant(P->groups.back()));
    for (size_t gi = 0; gi < P->groups.size(); ++gi) {
        const auto& g = P->groups[gi];
        const int v = chosen_variant(g);
        ScLaunch sl{g.dcases, g.djob[v], g.ncases, g.block[v], nullptr, overlap ? (int)SC_SKIP_IB : (int)SC_ALL,
                    dependent ? (int)(PDL_TRIGGER | PDL_DEPENDENT) : 0};
        int grid = overlap ? g.grid_overlap[v] : g.grid[v];
        if (fused) {
            for (const auto& lg : P->list_groups)
                if (lg.group == (int)gi) {
                    sl.list = lg.dlist[v];
                    sl.nlist = lg.n[v];
                }
            if (gi + 1 == P->groups.size()) {
                sl.echunks = P->dechunks32;
                sl.ecases = P->edge_groups[0].dcases;
                sl.nechunks = P->nechunks32;
                sl.count_cases = P->dcases_all;
                sl.ncount = (int)P->ctxs.size();
                sl.done = P->ddone;
            }
            // tail CTAs: one segment or edge chunk per warp
            const long long tail_jobs = sl.nlist + sl.nechunks;
            const int wpc = (g.block[v] > 0 ? g.block[v] : kThreads) / 32;
            sl.tail_ctas = tail_jobs > 0 ? (int)std::max<long long>(1, (tail_jobs + wpc - 1) / wpc) : 0;
            grid += sl.tail_ctas;
        }
        if (serial_tail && gi + 1 == P->groups.size()) {
            sl.phase = SC_ALL_TAIL;
            sl.echunks = P->dechunks32;
            sl.ecases = P->edge_groups[0].dcases;
            sl.nechunks = P->nechunks32;
            sl.count_cases = P->dcases_all;
            sl.ncount = (int)P->ctxs.size();
            sl.done = P->ddone;
            const int wpc = (g.block[v] > 0 ? g.block[v] : kThreads) / 32;
            sl.tail_ctas = sl.nechunks > 0 ? (int)std::max<long long>(1, (sl.nechunks + wpc - 1) / wpc) : 0;
            // the first phase leaves the tail CTAs' SMs free, so the edges run beside it
            const int per_sm = std::max(1, g.per_sm[v]);
            const int tail_sms = (sl.tail_ctas + per_sm - 1) / per_sm;
            grid = std::min<long long>(grid, (long long)std::max(1, P->sms - tail_sms) * per_sm) + sl.tail_ctas;
        }
        if ((e = timed_launch(timer, STAGE_SWEEP, st, [&] {
                 return launch_stream_collide(g.storage, g.collision, v, sl, g.jobs[v], grid, st);
             })) != cudaSuccess)
            return e;
    }
    if (fused || serial_tail) return cudaSuccess;
    // with one edge group the edge launch of the overlap order runs beside the IB-region
    // launches and advances the step counters itself
    const bool edges_end = overlap && P->edge_groups.size() == 1 && P->ddone;
    if (overlap)
        for (size_t k = 0; k < P->list_groups.size(); ++k) {
            const auto& lg = P->list_groups[k];
            // the same variant (segment width) as the group's sweep, so that every node sees
            // the same per-segment force decision as in the whole-lattice order
            const int v = chosen_variant(P->groups[lg.group]);
            const bool last = k + 1 == P->list_groups.size();
            ScLaunch sl{lg.dcases, nullptr, 0, 0, lg.dlist[v], (int)SC_LIST, (edges_end && last) ? (int)PDL_TRIGGER : 0};
            if ((e = launch_stream_collide(lg.storage, lg.collision, v, sl, lg.n[v], lg.grid[v], st)) != cudaSuccess)
                return e;
        }
    if (early) cudaStreamWaitEvent(st, P->ev_edges, 0);   // join before the step counters advance
    else if ((e = launch_edge_groups(P, st, timer, 0, edges_end)) != cudaSuccess) return e;
    if (edges_end) return cudaSuccess;
    return timed_launch(timer, STAGE_COUNTER, st, [&] { return launch_counters(P->dcases_all, (int)P->ctxs.size(), st); });
}

// IB-region segment lists of an overlap plan: footprints are built at the bodies'
// (fixed) markers, the boxes read back and every segment of the kIbAlign-aligned regions
// listed once per lattice, for each scalar variant's segment width.  Leaves overlap_ok false when a body is not fixed
// or has no footprint.
// At most this many IB CTAs (bodies) for the overlap: each holds a whole SM that the
// sweep beside it gives up (so all the sweep's CTAs run at once and its static job
// split stays balanced); beyond that the SMs given up cost more than the overlap saves.
constexpr int kOverlapMaxBodies = 8;
constexpr int kOverlapIbSms = 16;

int build_ib_lists(BatchPlan* P, int sms) {
    P->overlap_ok = false;
    if (P->ib_groups.size() != 1 || P->ib_groups[0].nrefs > kOverlapMaxBodies) return IBLBM_OK;
    for (auto* c : P->ctxs)
        for (auto& b : c->bodies)
            if (b.motion != MOT_FIXED) return IBLBM_OK;
    // small plans are latency-bound: the IB stage and the lattice edges then overlap better
    // the other way (edges beside the IB stage, the sweep after both)
    long long nodes = 0;
    for (auto* c : P->ctxs) nodes += (long long)c->hc.nx * c->hc.ny;
    if (nodes < kLargeGroupNodes) return IBLBM_OK;
    // the IB launch holds one SM per CTA (nrefs clusters of `cluster` CTAs), SMs the sweep
    // beside it gives up: at most kOverlapIbSms of them
    P->ib_groups[0].cluster = ib_cluster_size(P->ib_groups[0].storage, P->ib_groups[0].nrefs, kOverlapIbSms);
    const int free_sms = sms - P->ib_groups[0].nrefs * std::max(1, P->ib_groups[0].cluster);
    for (auto& g : P->groups)
        for (int v = 0; v < SC_VARIANTS; ++v) {
            const long long cap = (long long)free_sms * sc_blocks_per_sm(g.storage, g.collision, v);
            g.grid_overlap[v] = (int)std::max<long long>(1, std::min<long long>((g.jobs[v] + 7) / 8, cap));
            if (g.block[v] == 64)
                g.grid_overlap[v] = (int)std::max<long long>(1, std::min<long long>((g.jobs[v] + 1) / 2, 4 * cap));
        }
    for (auto& g : P->ib_groups) {
        IbLaunch setup{g.drefs, g.nrefs, 1, 0, 0};
        int rc = check(launch_ib(g.storage, setup, P->st));
        if (rc) return rc;
    }
    int rc = check(cudaStreamSynchronize(P->st));
    if (rc) return rc;
    for (size_t gi = 0; gi < P->groups.size(); ++gi) {
        const auto& grp = P->groups[gi];
        ListGroup lg;
        lg.storage = grp.storage;
        lg.collision = grp.collision;
        lg.group = (int)gi;
        lg.dcases = grp.dcases;
        bool any = false;
        for (int v : {(int)SC_SCALAR, (int)SC_SCALAR2}) {
            std::vector<int4> list;
            const int seg = sc_segment(grp.storage, v);
            int ci = 0;
            for (auto* c : P->ctxs) {
                if (c->hc.storage != grp.storage || c->hc.collision != grp.collision) continue;
                std::set<std::pair<int, int>> segs;
                for (int b = 0; b < (int)c->bodies.size(); ++b) {
                    BodyDev B;
                    if (cudaMemcpy(&B, &c->dbodies[b], sizeof(BodyDev), cudaMemcpyDeviceToHost) != cudaSuccess)
                        return check(cudaGetLastError());
                    if (B.nfp <= 0) return IBLBM_OK;
                    for (int y = B.by0; y < B.by0 + B.bh; ++y)
                        for (int x = 0; x < c->hc.nx; x += seg)
                            if (in_ib_region(y, x, B.bx0, B.by0, B.bw, B.bh)) segs.insert({y, x});
                }
                for (auto& sg : segs) list.push_back(make_int4(ci, sg.first, sg.second, 0));
                ++ci;
            }
            if (list.empty()) continue;
            any = true;
            lg.n[v] = (long long)list.size();
            lg.grid[v] = (int)std::max<long long>(1, std::min<long long>((lg.n[v] + 15) / 16, 4LL * sms));
            lg.dlist[v] = static_cast<int4*>(plan_alloc(P, sizeof(int4) * list.size()));
            if (!lg.dlist[v]) return IBLBM_ERR_OOM;
            cudaMemcpyAsync(lg.dlist[v], list.data(), sizeof(int4) * list.size(), cudaMemcpyHostToDevice, P->st);
        }
        if (any) P->list_groups.push_back(lg);
    }
    rc = check(cudaStreamSynchronize(P->st));
    if (rc) return rc;
    P->overlap_ok = true;
    return IBLBM_OK;
}

BatchPlan* get_plan(iblbm_ctx** ctxs, int n, int* rc) {
    std::vector<iblbm_ctx*> key(ctxs, ctxs + n);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        bool ok = true;
        for (int i = 0; i < n; ++i) ok &= it->second->versions[i] == ctxs[i]->version;
        if (ok) return it->second;
        delete it->second;
        g_plans.erase(it);
    }
    BatchPlan* P = new BatchPlan();
    P->ctxs = key;
    P->st = ctxs[0]->work;
    for (int i = 0; i < n; ++i) P->versions.push_back(ctxs[i]->version);
    std::vector<BodyRef> all_refs;
    std::vector<CaseDev*> all_cases;
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctxs[0]->device);
    P->sms = sms;
    for (int st = 0; st < 3; ++st) {
        std::vector<BodyRef> refs;
        for (int i = 0; i < n; ++i) {
            iblbm_ctx* c = ctxs[i];
            if (c->hc.storage != st) continue;
            all_cases.push_back(c->dc);
            for (int b = 0; b < (int)c->bodies.size(); ++b) refs.push_back(BodyRef{c->dc, &c->dbodies[b], b, 0});
        }
        if (!refs.empty()) {
            IbGroup ig;
            ig.storage = st;
            ig.nrefs = (int)refs.size();
            ig.cluster = ib_cluster_size(st, ig.nrefs, sms / 2);
            ig.drefs = static_cast<BodyRef*>(plan_alloc(P, sizeof(BodyRef) * refs.size()));
            if (!ig.drefs) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
            cudaMemcpyAsync(ig.drefs, refs.data(), sizeof(BodyRef) * refs.size(), cudaMemcpyHostToDevice, P->st);
            P->ib_groups.push_back(ig);
            all_refs.insert(all_refs.end(), refs.begin(), refs.end());
        }
        {
            EdgeGroup eg;
            eg.storage = st;
            std::vector<CaseDev*> cs;
            std::vector<EdgeChunk> chunks;
            // chunk size: kThreads nodes, smaller when that would leave SMs idle (the edge
            // work of one small lattice is compute-bound in FP64 and should spread out)
            long long total = 0;
            for (int i = 0; i < n; ++i)
                if (ctxs[i]->hc.storage == st) total += lattice_edge_nodes(ctxs[i]->hc.nx, ctxs[i]->hc.ny);
            int chunk = (int)std::min<long long>(kThreads, (total + 2LL * sms - 1) / (2LL * sms));
            chunk = std::max(32, (chunk + 31) / 32 * 32);
            eg.block = chunk;
            for (int i = 0; i < n; ++i) {
                iblbm_ctx* c = ctxs[i];
                if (c->hc.storage != st) continue;
                const int ne = (int)lattice_edge_nodes(c->hc.nx, c->hc.ny);
                for (int f = 0; f < ne; f += chunk) chunks.push_back(EdgeChunk{(int)cs.size(), f, std::min(ne, f + chunk), 0});
                cs.push_back(c->dc);
            }
            if (!cs.empty()) {
                eg.nchunks = (int)chunks.size();
                eg.dcases = static_cast<CaseDev**>(plan_alloc(P, sizeof(CaseDev*) * cs.size()));
                eg.dchunks = static_cast<EdgeChunk*>(plan_alloc(P, sizeof(EdgeChunk) * chunks.size()));
                if (!eg.dcases || !eg.dchunks) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
                cudaMemcpyAsync(eg.dcases, cs.data(), sizeof(CaseDev*) * cs.size(), cudaMemcpyHostToDevice, P->st);
                cudaMemcpyAsync(eg.dchunks, chunks.data(), sizeof(EdgeChunk) * chunks.size(), cudaMemcpyHostToDevice,
                                P->st);
                P->edge_groups.push_back(eg);
            }
        }
        for (int col = 0; col < 4; ++col) {
            BatchGroup g;
            g.storage = st;
            g.collision = col;
            std::vector<CaseDev*> cs;
            for (int i = 0; i < n; ++i) {
                iblbm_ctx* c = ctxs[i];
                if (c->hc.storage == st && c->hc.collision == col) cs.push_back(c->dc);
            }
            if (cs.empty()) continue;
            g.ncases = (int)cs.size();
            g.dcases = static_cast<CaseDev**>(plan_alloc(P, sizeof(CaseDev*) * cs.size()));
            if (!g.dcases) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
            cudaMemcpyAsync(g.dcases, cs.data(), sizeof(CaseDev*) * cs.size(), cudaMemcpyHostToDevice, P->st);
            long long group_nodes = 0;
            for (int i = 0; i < n; ++i)
                if (ctxs[i]->hc.storage == st && ctxs[i]->hc.collision == col)
                    group_nodes += (long long)ctxs[i]->hc.nx * ctxs[i]->hc.ny;
            g.size_class = group_nodes >= kLargeGroupNodes ? 1 : 0;
            for (int v = 0; v < SC_VARIANTS; ++v) {
                const int seg = sc_segment(st, v);
                std::vector<long long> off{0};
                g.ok[v] = true;
                for (int i = 0; i < n; ++i) {
                    iblbm_ctx* c = ctxs[i];
                    if (c->hc.storage == st && c->hc.collision == col) {
                        off.push_back(off.back() + (long long)c->hc.ny * ((c->hc.nx + seg - 1) / seg));
                        g.ok[v] = g.ok[v] && sc_variant_ok(v, c->hc.f[0], c->hc.f[1]);
                    }
                }
                g.jobs[v] = off.back();
                g.djob[v] = static_cast<long long*>(plan_alloc(P, sizeof(long long) * off.size()));
                if (!g.djob[v]) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
                cudaMemcpyAsync(g.djob[v], off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, P->st);
                const long long cap = (long long)sms * sc_blocks_per_sm(st, col, v);
                g.per_sm[v] = (int)(cap / sms);
                g.grid[v] = (int)std::max<long long>(1, std::min<long long>((g.jobs[v] + 7) / 8, cap));
                if ((v == SC_SCALAR || v == SC_SCALAR2) && (g.jobs[v] + 7) / 8 < sms) {
                    // too few jobs to give every SM a 256-thread CTA: spread 64-thread CTAs
                    g.block[v] = 64;
                    g.per_sm[v] = (int)(4 * cap / sms);
                    g.grid[v] = (int)std::max<long long>(1, std::min<long long>((g.jobs[v] + 1) / 2, 4 * cap));
                }
            }
            P->groups.push_back(g);
        }
    }
    P->ddone = static_cast<unsigned*>(plan_alloc(P, sizeof(unsigned)));
    if (!P->ddone) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
    cudaMemsetAsync(P->ddone, 0, sizeof(unsigned), P->st);
    // one storage type: the lattice edges in 32-node chunks (one warp each), in the order of
    // the edge group's cases, for the tail of the last sweep launch
    if (P->edge_groups.size() == 1 && P->ddone) {
        std::vector<EdgeChunk> chunks;
        int ci = 0;
        for (auto* c : P->ctxs) {
            if (c->hc.storage != P->edge_groups[0].storage) continue;
            const int ne = (int)lattice_edge_nodes(c->hc.nx, c->hc.ny);
            for (int f = 0; f < ne; f += 32) chunks.push_back(EdgeChunk{ci, f, std::min(ne, f + 32), 0});
            ++ci;
        }
        if (!chunks.empty()) {
            P->dechunks32 = static_cast<EdgeChunk*>(plan_alloc(P, sizeof(EdgeChunk) * chunks.size()));
            if (!P->dechunks32) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
            cudaMemcpyAsync(P->dechunks32, chunks.data(), sizeof(EdgeChunk) * chunks.size(), cudaMemcpyHostToDevice,
                            P->st);
            P->nechunks32 = (int)chunks.size();
            P->fused_tail = true;
        }
    }
    P->nrefs_all = (int)all_refs.size();
    P->drefs_all = static_cast<BodyRef*>(plan_alloc(P, sizeof(BodyRef) * std::max<size_t>(1, all_refs.size())));
    P->dcases_all = static_cast<CaseDev**>(plan_alloc(P, sizeof(CaseDev*) * all_cases.size()));
    if (!P->drefs_all || !P->dcases_all) { *rc = IBLBM_ERR_OOM; delete P; return nullptr; }
    if (!all_refs.empty())
        cudaMemcpyAsync(P->drefs_all, all_refs.data(), sizeof(BodyRef) * all_refs.size(), cudaMemcpyHostToDevice, P->st);
    cudaMemcpyAsync(P->dcases_all, all_cases.data(), sizeof(CaseDev*) * all_cases.size(), cudaMemcpyHostToDevice, P->st);
    for (int i = 0; i < n; ++i) {
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        P->joins.push_back(e);
    }
    *rc = check(cudaStreamSynchronize(P->st));
    if (*rc) { delete P; return nullptr; }
    // autotune: time each variant of every group whose (storage, collision) has no choice yet
    for (auto& g : P->groups) {
        if (g_variant[g.storage][g.collision][g.size_class] >= 0) continue;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        int best = SC_SCALAR;
        double best_ms = 1e300;
        for (int v = 0; v < SC_VARIANTS; ++v) {
            if (!g.ok[v]) {
                g_variant_ms[g.storage][g.collision][g.size_class][v] = 0.0;
                continue;
            }
            ScLaunch sl{g.dcases, g.djob[v], g.ncases, g.block[v], nullptr, (int)SC_ALL, 0};
            float ms = 0.f, tot = 0.f;
            launch_stream_collide(g.storage, g.collision, v, sl, g.jobs[v], g.grid[v], P->st);   // warm
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(a, P->st);
                launch_stream_collide(g.storage, g.collision, v, sl, g.jobs[v], g.grid[v], P->st);
                cudaEventRecord(b, P->st);
                cudaEventSynchronize(b);
                cudaEventElapsedTime(&ms, a, b);
                tot += ms;
            }
            g_variant_ms[g.storage][g.collision][g.size_class][v] = tot / 3.0;
            if (tot / 3.0 < best_ms) {
                best_ms = tot / 3.0;
                best = v;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        // the one- and two-node-per-lane sweeps can run beside the IB stage: keep the fastest
        // of them unless another variant is clearly faster on its own
        int best_phased = -1;
        for (int v = 0; v < SC_VARIANTS; ++v)
            if (sc_variant_phased(v) && g.ok[v] &&
                (best_phased < 0 || g_variant_ms[g.storage][g.collision][g.size_class][v] <
                                        g_variant_ms[g.storage][g.collision][g.size_class][best_phased]))
                best_phased = v;
        if (best_phased >= 0 && !sc_variant_phased(best) &&
            g_variant_ms[g.storage][g.collision][g.size_class][best_phased] < 1.1 * best_ms)
            best = best_phased;
        g_variant[g.storage][g.collision][g.size_class] = best;
    }
    // edge launch overlapped with the IB stage when no footprint can reach a lattice
    // edge: every body fixed where it was added, its markers (within `reach` of the
    // centre) plus the Peskin stencil and a margin clear of the edge rows and columns
    bool clear = true;
    for (int i = 0; i < n; ++i)
        for (const auto& b : ctxs[i]->bodies) {
            const double m = b.reach + 4.0;
            clear = clear && b.motion == MOT_FIXED && !b.moved && b.xc - m > 1.0 && b.yc - m > 1.0 &&
                    b.xc + m < ctxs[i]->hc.nx - 2.0 && b.yc + m < ctxs[i]->hc.ny - 2.0;
        }
    if (clear && !P->edge_groups.empty()) {
        if (cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_edges, cudaEventDisableTiming) != cudaSuccess) {
            *rc = IBLBM_ERR_CUDA;
            delete P;
            return nullptr;
        }
        P->edges_early = true;
    }
    *rc = check(cudaStreamSynchronize(P->st));
    if (*rc) { delete P; return nullptr; }
    for (int i = 0; i < n; ++i) {
        int ndfc = 0;
        bool moving = false;
        for (const auto& b : ctxs[i]->bodies)
            if (b.scheme == SCH_DFC) {
                ++ndfc;
                moving = moving || b.motion != MOT_FIXED;
            }
        if (ndfc >= 2 && moving) P->prepare_first = true;
    }
    *rc = build_ib_lists(P, sms);
    if (*rc) { delete P; return nullptr; }
    g_plans[key] = P;
    return P;
}

int batch_capture(BatchPlan* P, int nsteps, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return check(e);
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) e = launch_batch_step(P, P->st, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(P->st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return check(e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return check(e);
}

}  // namespace

extern "C" int iblbm_set_kernel_variant(int storage, int collision, int variant) {
    if (storage < 0 || storage > 2 || collision < 0 || collision > 3 || variant < -1 || variant >= SC_VARIANTS)
        return IBLBM_ERR_INVALID_ARG;
    g_variant[storage][collision][0] = g_variant[storage][collision][1] = variant;
    for (auto& kv : g_plans) kv.second->graphs.reset();   // captured graphs hold the old kernel
    return IBLBM_OK;
}

extern "C" int iblbm_test_set_consumer_poll_limit(long polls) {
    if (cudaDeviceSynchronize() != cudaSuccess || set_consumer_poll_limit(polls) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    return IBLBM_OK;
}

extern "C" int iblbm_test_set_ib_fast(int enable) {
    if (cudaDeviceSynchronize() != cudaSuccess || set_ib_fast(enable) != cudaSuccess) {
        cudaGetLastError();
        return IBLBM_ERR_CUDA;
    }
    return IBLBM_OK;
}

extern "C" int iblbm_kernel_variant(int storage, int collision, int* variant, double* ms) {
    if (storage < 0 || storage > 2 || collision < 0 || collision > 3) return IBLBM_ERR_INVALID_ARG;
    const int cls = g_variant[storage][collision][1] >= 0 ? 1 : 0;   // the large class when tuned
    if (variant) *variant = g_variant[storage][collision][cls];
    if (ms)
        for (int v = 0; v < SC_VARIANTS; ++v) ms[v] = g_variant_ms[storage][collision][cls][v];
    return IBLBM_OK;
}

extern "C" int iblbm_step_batch(iblbm_ctx** ctxs, int n, int nsteps) {
    return iblbm_internal_step_batch(ctxs, n, nsteps, 1);
}

int iblbm_internal_step_batch(iblbm_ctx** ctxs, int n, int nsteps, int use_graphs) {
    if (!ctxs || n <= 0 || nsteps < 0) return IBLBM_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || ctxs[i]->device != ctxs[0]->device) return IBLBM_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return IBLBM_ERR_INVALID_ARG;
    }
    if (nsteps == 0) return IBLBM_OK;
    int rc = IBLBM_OK;
    BatchPlan* P = get_plan(ctxs, n, &rc);
    if (!P) return rc;
    iblbm_ctx* lead = ctxs[0];
    // order after every context's own stream and previous work
    for (int i = 0; i < n; ++i) {
        begin_user(ctxs[i]);
        if (i > 0) {
            cudaEventRecord(P->joins[i], ctxs[i]->work);
            cudaStreamWaitEvent(P->st, P->joins[i], 0);
        }
    }
    if (lead->timing || !use_graphs) {
        for (int s = 0; s < nsteps && !rc; ++s) rc = check(launch_batch_step(P, P->st, lead->timing ? lead : nullptr));
    } else {
        if (!P->graphs.one) {
            rc = batch_capture(P, 1, &P->graphs.one);
            if (!rc) {
                P->graphs.many_steps = 8;
                rc = batch_capture(P, P->graphs.many_steps, &P->graphs.many);
            }
        }
        int left = nsteps;
        while (!rc && left >= P->graphs.many_steps) {
            rc = check(cudaGraphLaunch(P->graphs.many, P->st));
            left -= P->graphs.many_steps;
        }
        while (!rc && left > 0) {
            rc = check(cudaGraphLaunch(P->graphs.one, P->st));
            --left;
        }
    }
    cudaEventRecord(P->joins[0], P->st);
    for (int i = 0; i < n; ++i) {
        if (i > 0) cudaStreamWaitEvent(ctxs[i]->work, P->joins[0], 0);
        end_user(ctxs[i]);
        if (!rc) ctxs[i]->steps += nsteps;
    }
    return rc;
}

// Drops cached batch plans that contain a context about to be destroyed.
static void forget_plans(iblbm_ctx* c) {
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (std::find(it->first.begin(), it->first.end(), c) != it->first.end()) {
            cudaStreamSynchronize(it->second->st);
            delete it->second;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}
