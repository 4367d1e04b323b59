// Device-side data structures and per-node arithmetic of the IB-LBM path.
//
// Populations are stored shifted, s_i = f_i - w_i, one plane per direction with
// a row pitch that is a multiple of 32 elements (16-byte aligned rows for every
// storage type).  All node arithmetic below works on shifted values so that FP32
// and FP16 storage keep the small deviations from rest at full relative precision.
#pragma once

#ifdef IBLBM_EMULATE
#include "cuda_emu.h"   // host-thread emulation used only by the CPU test suite
#else
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#define IBLBM_LAUNCH(kern, grid, block, stream, ...) kern<<<(grid), (block), 0, (stream)>>>(__VA_ARGS__)
#define IBLBM_LAUNCH_SMEM(kern, grid, block, smem, stream, ...) \
    kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__)
#define IBLBM_DYNAMIC_SMEM(name) extern __shared__ __align__(128) unsigned char name[]
// Launch that may begin before the previous kernel of the stream ends (programmatic
// dependent launch) when `dependent` is true; a plain launch otherwise.
#define IBLBM_LAUNCH_PDL(kern, grid, block, strm_, dependent, ...)                                  \
    do {                                                                                           \
        cudaLaunchConfig_t cfg_ = {};                                                              \
        cfg_.gridDim = dim3(grid);                                                                 \
        cfg_.blockDim = dim3(block);                                                               \
        cfg_.dynamicSmemBytes = 0;                                                                 \
        cfg_.stream = (strm_);                                                                     \
        cudaLaunchAttribute at_[1];                                                                \
        at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                            \
        at_[0].val.programmaticStreamSerializationAllowed = 1;                                     \
        cfg_.attrs = at_;                                                                          \
        cfg_.numAttrs = (dependent) ? 1 : 0;                                                       \
        cudaLaunchKernelEx(&cfg_, kern, __VA_ARGS__);                                              \
    } while (0)
#endif
#include <stdint.h>

namespace iblbm {

// ---- enums (values match include/iblbm.h) -----------------------------------------
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2 };
enum { BC_PER = 0, BC_VEL = 1, BC_NEU = 2 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };
enum { COL_BGK = 0, COL_TRT = 1, COL_CM = 2, COL_NONE = 3 };
enum { K_HAT = 0, K_P4 = 1 };
enum { SCH_DF = 0, SCH_MDF = 1, SCH_DFC = 2 };
enum { MOT_FIXED = 0, MOT_PRESC = 1, MOT_FREE = 2, MOT_FREE_TRANSLATION = 3 };
// device status bits
enum : unsigned {
    STAT_UNSTABLE = 1u,
    STAT_MARKER_OUT = 2u,
    STAT_CAPACITY = 4u,
    STAT_MDF_WARN = 8u,
    STAT_TIMEOUT = 16u,   // a bounded device-side wait gave up
};

constexpr int kMaxBodies = 64;   // bodies per lattice
constexpr int kThreads = 256;    // threads per CTA of every kernel here

struct BodyDev;

// One lattice (case) in device memory.
struct CaseDev {
    int nx, ny, pitch, storage;
    long long plane;              // elements per population plane (pitch * ny)
    int collision;
    int bc[4];
    double ubc[4][2];
    double tau, omega, s_e, s_o, cm_sq, cm_se;
    double gfx, gfy;
    void* f[2];                   // A/B population buffers; step parity selects the source
    int nbodies;
    int dfc_all_fixed;            // 1: DFC lambda_k can be cached
    BodyDev* bodies;              // device array [kMaxBodies]
    unsigned long long step;
    unsigned int status;
    int wall_bb;                  // bit s: side s closes by on-node bounce-back (wall_closure = 1 and a
                                  // zero velocity, decided once on the host from the FP64 u_bc)
    int n_mdf, mdf_lead;          // MDF bodies; with two or more they iterate coupled, stepped by
                                  // the IB CTA of the first (mdf_lead)
    void* cpl;                    // coupled MDF scratch, 3 nx ny R: spread F_x, F_y, 1/(2 rho) per node
};

// Dynamic FP64 state of a rigid body (what a checkpoint carries besides arrays).
struct BodyState {
    double xc, yc, vx, vy, om, theta;       // after the last step
    double Fhx, Fhy, Th, dFimx, dFimy;       // force/torque of the last step, Eq. A3 increment
    double vhx, vhy, omh;                    // half-step velocities of the step in flight
    double mdf_omega, mdf_res;
    long long nstep, hist_n;
    int mdf_iters, omega_valid;
    double mdf_omega_end;                    // relaxation in use when the last MDF iteration ended
};

// One rigid body in device memory (R-typed scratch as void*).
struct BodyDev {
    int n, kernel, scheme, motion, internal_mass, mdf_nmin, mdf_nmax, S;
    double ds, radius, rho_ratio, gx, gy, mdf_tol, osc_amp, osc_period, xc0, yc0;
    long long t0;                 // case step at which the body was added
    BodyState st;
    // markers
    double *X, *Y, *r0x, *r0y, *Udx, *Udy, *Fx, *Fy, *lam;
    // footprint: bounding box, box-local node -> slot map, node CSR over markers
    int bx0, by0, bw, bh, box_cap, nfp, nent, cache_valid, lam_valid;
    int ud_given;                 // FIXED: U_d set per marker by the caller, not v + omega x r
    int ud_current;               // FIXED: U_d already holds v + omega x r (set on the device, cleared by
                                  // every host write of the body)
    int* node_map;                // [box_cap]
    int* fp_node;                 // [nent] slot -> box-local node
    int* csr_off;                 // [nent + 1]
    int* csr_ent;                 // [nent] entry = k*S*S + b*S + a, sorted by k per slot
    int* fill;                    // [nent]
    void* csr_w;                  // [nent] kernel weight D of each CSR entry (R)
    int* mslot;                   // [nent] footprint slot of stencil node r of marker k (k S^2 + r)
    int* ij;                      // [2n] stencil origins
    void* wts;                    // [n][8] kernel weights phi_x[4], phi_y[4] (R)
    void* fpdata;                 // [nent][9] gathered slot data (R)
    void* patch;                  // [nent][9] spread result consumed by stream-collide (R)
    void* mk;                     // [n][16] marker scratch (R)
    double* hist;                 // [hist_cap][3]
    int hist_cap;
    unsigned int status;
};

// ---- D2Q9 lattice (Sec. 2.1) ---------------------------------------------------------
__host__ __device__ constexpr int ex(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int ey(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 5 + 2) % 4) + 5); }
template <class R>
__host__ __device__ constexpr R wgt(int i) { return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36)); }

// ---- storage traits: 16-byte vectors ------------------------------------------------
template <class S> struct Traits;
// V: nodes per 16-byte vector; kMinBlocks: resident 256-thread CTAs per SM the
// stream-collide kernel is compiled for (register budget 65536 / (256 kMinBlocks)).
template <> struct Traits<double> { using R = double; static constexpr int V = 2; static constexpr int kMinBlocks = 1; };
template <> struct Traits<float> { using R = float; static constexpr int V = 4; static constexpr int kMinBlocks = 3; };
template <> struct Traits<__half> { using R = float; static constexpr int V = 8; static constexpr int kMinBlocks = 2; };

template <class R> __device__ __forceinline__ R to_r(double v) { return R(v); }

__device__ __forceinline__ double ld1(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __half* p) { return __half2float(__ldg(p)); }

// Read-only load for the stream-collide sweep, which reads whole rows of every plane:
// FP32 asks L2 to fetch 256-byte blocks around each miss.
__device__ __forceinline__ double ld1_sweep(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld1_sweep(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld1_sweep(const float* p) {
#ifdef IBLBM_EMULATE
    return *p;
#else
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
#endif
}

// The same loads with an L2 evict-first hint, for the sweep that runs beside the IB
// stage: the streamed planes then give way in L2 before the IB stage's code and data.
__device__ __forceinline__ double ld1_sweep_ef(const double* p) {
#ifdef IBLBM_EMULATE
    return *p;
#else
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
#endif
}
__device__ __forceinline__ float ld1_sweep_ef(const float* p) {
#ifdef IBLBM_EMULATE
    return *p;
#else
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    float v;
    asm("ld.global.nc.L2::cache_hint.L2::256B.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
#endif
}
__device__ __forceinline__ float ld1_sweep_ef(const __half* p) { return ld1_sweep(p); }

// FP16 storage, two adjacent nodes per 32-bit word (the pair sweep): read-only load
// with the same 256-byte L2 fetch as the FP32 sweep, the unpacking to FP32, and the
// store of two correctly rounded values.
__device__ __forceinline__ unsigned ld2h_sweep(const __half* p) {
#ifdef IBLBM_EMULATE
    unsigned v;
    std::memcpy(&v, p, 4);
    return v;
#else
    unsigned v;
    asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
#endif
}
__device__ __forceinline__ float2 unpack2h(unsigned v) {
    __half2_raw r;
    r.x = (unsigned short)(v & 0xffffu);
    r.y = (unsigned short)(v >> 16);
    return __half22float2(__half2(r));
}
__device__ __forceinline__ void st2h(__half* p, float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    const __half2_raw r = h;
    *reinterpret_cast<unsigned*>(p) = (unsigned)r.x | ((unsigned)r.y << 16);
}

__device__ __forceinline__ void st1(double* p, double v) { *p = v; }
__device__ __forceinline__ void st1(float* p, float v) { *p = v; }
__device__ __forceinline__ void st1(__half* p, float v) { *p = __float2half_rn(v); }
// Store of the stream-collide sweep (the destination is not read again this step).
__device__ __forceinline__ void st1_sweep(double* p, double v) { st1(p, v); }
__device__ __forceinline__ void st1_sweep(__half* p, float v) { st1(p, v); }
__device__ __forceinline__ void st1_sweep(float* p, float v) { *p = v; }
// Store with an L2 evict-last hint: the IB-region populations written at the end of a
// step are the ones the next step's IB stage gathers first, while the sweep beside it
// streams the rest of the lattice through L2.
__device__ __forceinline__ void st1_keep(double* p, double v) {
#ifdef IBLBM_EMULATE
    *p = v;
#else
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
#endif
}
__device__ __forceinline__ void st1_keep(float* p, float v) {
#ifdef IBLBM_EMULATE
    *p = v;
#else
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
#endif
}
__device__ __forceinline__ void st1_keep(__half* p, float v) { st1(p, v); }
// One correctly rounded conversion from double (no double rounding through float).
__device__ __forceinline__ void st1_from_double(double* p, double v) { *p = v; }
__device__ __forceinline__ void st1_from_double(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void st1_from_double(__half* p, double v) { *p = __double2half(v); }

__device__ __forceinline__ void ld16(const double* p, double (&v)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2*>(p));
    v[0] = t.x; v[1] = t.y;
}
__device__ __forceinline__ void ld16(const float* p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
union Half8 {   // 16 bytes viewed as four half pairs (union punning, no aliasing casts)
    uint4 u;
    __half2 h[4];
};
__device__ __forceinline__ void ld16(const __half* p, float (&v)[8]) {
    Half8 t;
    t.u = __ldg(reinterpret_cast<const uint4*>(p));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __half22float2(t.h[k]);
        v[2 * k] = f.x; v[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void st16(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void st16(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st16(__half* p, const float (&v)[8]) {
    Half8 t;
#pragma unroll
    for (int k = 0; k < 4; ++k) t.h[k] = __floats2half2_rn(v[2 * k], v[2 * k + 1]);
    *reinterpret_cast<uint4*>(p) = t.u;
}

// ---- collision parameters held in registers ------------------------------------------
template <class R>
struct CollParams {
    int kind;
    R omega, s_e, s_o, sq, se;
    __device__ __forceinline__ void load(const CaseDev& c) {
        kind = c.collision;
        omega = R(c.omega); s_e = R(c.s_e); s_o = R(c.s_o); sq = R(c.cm_sq); se = R(c.cm_se);
    }
};

// Shifted equilibrium seq_i = f_i^eq - w_i (Eq. 2) at density rho = 1 + drho.
template <class R>
__device__ __forceinline__ R seq_i(int i, R drho, R rho, R ux, R uy, R uu) {
    R eu = R(ex(i)) * ux + R(ey(i)) * uy;
    return wgt<R>(i) * (drho + rho * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu));
}

// Bracket of Eq. 3 without the prefactor: w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)].
template <class R>
__device__ __forceinline__ R guo_i(int i, R ux, R uy, R Fx, R Fy) {
    R eu = R(ex(i)) * ux + R(ey(i)) * uy;
    R eF = R(ex(i)) * Fx + R(ey(i)) * Fy;
    return wgt<R>(i) * (R(3) * ((R(ex(i)) - ux) * Fx + (R(ey(i)) - uy) * Fy) + R(9) * eu * eF);
}

// 1-D moment shifts used by the central-moment operator (raw <-> central about u).
template <class R>
__device__ __forceinline__ void to_central(R& c0, R& c1, R& c2, R u) {
    R r0 = c0, r1 = c1, r2 = c2;
    c1 = r1 - u * r0;
    c2 = r2 - R(2) * u * r1 + u * u * r0;
}
template <class R>
__device__ __forceinline__ void to_raw(R& c0, R& c1, R& c2, R u) {
    R k0 = c0, k1 = c1, k2 = c2;
    c1 = k1 + u * k0;
    c2 = k2 + R(2) * u * k1 + u * u * k0;
}

// Collide one node in place on shifted populations.  F is the force density
// acting at the node (Guo forcing, Eq. 3-4; TRT split source; CM-MRT source R).
// Returns rho for the stability check.
// KIND >= 0 fixes the operator at compile time (specialised kernels); -1 reads it from P.
// FORCED = false drops every force term (nodes with F = 0 exactly), saving issue slots.

template <class R, bool FORCED>
__device__ __forceinline__ R collide_cm(const CollParams<R>& P, R (&s)[9], R Fx, R Fy) {
    // Central-moment MRT (Eq. 5) on the deviation from rest.  With k(f) the
    // central moments about u and f = w + s:
    //   s* = T^-1 [ (I - L) k(s) + L (k_eq - k(w)) + (I - L/2) R ],
    // where k(w) are the central moments of the rest weights (closed form).
    // Raw moments use the tensor-product structure of D2Q9 (velocity
    // components in {-1, 0, 1}); central moments follow by 1-D binomial shifts.
    // Population index by (cx, cy): row cy=0 -> (3, 0, 1), cy=1 -> (6, 2, 5), cy=-1 -> (7, 4, 8).
    R m[3][3];   // m[p][q] = sum s cx^p cy^q
    {
        R a0 = s[3] + s[0] + s[1], b0 = s[1] - s[3], c0 = s[1] + s[3];
        R a1 = s[6] + s[2] + s[5], b1 = s[5] - s[6], c1 = s[5] + s[6];
        R a2 = s[7] + s[4] + s[8], b2 = s[8] - s[7], c2 = s[8] + s[7];   // cy = -1
        m[0][0] = a0 + a1 + a2; m[0][1] = a1 - a2; m[0][2] = a1 + a2;
        m[1][0] = b0 + b1 + b2; m[1][1] = b1 - b2; m[1][2] = b1 + b2;
        m[2][0] = c0 + c1 + c2; m[2][1] = c1 - c2; m[2][2] = c1 + c2;
    }
    // density and momentum are among these raw moments (m00 = drho, m10 = j_x, m01 = j_y)
    const R drho = m[0][0];
    const R rho = R(1) + drho;
    const R inv = R(1) / rho;
    const R ux = (FORCED ? m[1][0] + R(0.5) * Fx : m[1][0]) * inv;   // Eq. 4
    const R uy = (FORCED ? m[0][1] + R(0.5) * Fy : m[0][1]) * inv;
    const R uu = ux * ux + uy * uy;
#pragma unroll
    for (int q = 0; q < 3; ++q) to_central(m[0][q], m[1][q], m[2][q], ux);
#pragma unroll
    for (int p = 0; p < 3; ++p) to_central(m[p][0], m[p][1], m[p][2], uy);
    const R cs2 = R(1) / R(3), cs4 = R(1) / R(9);
    const R ux2 = ux * ux, uy2 = uy * uy;
    const R w = P.omega;
    // second order: k20, k02, k11 relax with omega
    R k20 = (R(1) - w) * m[2][0] + w * (drho * cs2 - ux2);
    R k02 = (R(1) - w) * m[0][2] + w * (drho * cs2 - uy2);
    R k11 = (R(1) - w) * m[1][1] + w * (-ux * uy);
    // third order: k21, k12 relax with s_q, source cs2 F
    R k21 = (R(1) - P.sq) * m[2][1] + P.sq * (uy * (cs2 + ux2));
    R k12 = (R(1) - P.sq) * m[1][2] + P.sq * (ux * (cs2 + uy2));
    if (FORCED) {
        k21 += (R(1) - R(0.5) * P.sq) * cs2 * Fy;
        k12 += (R(1) - R(0.5) * P.sq) * cs2 * Fx;
    }
    // fourth order: k22 relaxes with s_e
    R k22 = (R(1) - P.se) * m[2][2] + P.se * (drho * cs4 - cs2 * uu - ux2 * uy2);
    // conserved k00, and k10/k01 carry the full source (I - 0/2) R = F
    if (FORCED) {
        m[1][0] += Fx;
        m[0][1] += Fy;
    }
    m[2][0] = k20; m[0][2] = k02; m[1][1] = k11; m[2][1] = k21; m[1][2] = k12; m[2][2] = k22;
#pragma unroll
    for (int p = 0; p < 3; ++p) to_raw(m[p][0], m[p][1], m[p][2], uy);
#pragma unroll
    for (int q = 0; q < 3; ++q) to_raw(m[0][q], m[1][q], m[2][q], ux);
    // raw moments -> populations: g_q(0) = m0q - m2q, g_q(+1) = (m1q + m2q)/2, g_q(-1) = (m2q - m1q)/2
    R g[3][3];   // g[cxi][q], cxi: 0 -> cx=0, 1 -> cx=+1, 2 -> cx=-1
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        g[0][q] = m[0][q] - m[2][q];
        g[1][q] = R(0.5) * (m[1][q] + m[2][q]);
        g[2][q] = R(0.5) * (m[2][q] - m[1][q]);
    }
    // s(cx, cy) = h(cy) over q: cy=0 -> g0 - g2, cy=+1 -> (g1 + g2)/2, cy=-1 -> (g2 - g1)/2
    auto h0 = [&](int c) { return g[c][0] - g[c][2]; };
    auto hp = [&](int c) { return R(0.5) * (g[c][1] + g[c][2]); };
    auto hm = [&](int c) { return R(0.5) * (g[c][2] - g[c][1]); };
    s[0] = h0(0); s[1] = h0(1); s[3] = h0(2);
    s[2] = hp(0); s[5] = hp(1); s[6] = hp(2);
    s[4] = hm(0); s[8] = hm(1); s[7] = hm(2);
    return rho;
}

template <class R, int KIND = -1, bool FORCED = true>
__device__ __forceinline__ R collide(const CollParams<R>& P, R (&s)[9], R Fx, R Fy) {
    const int kind = KIND >= 0 ? KIND : P.kind;
    if (kind == COL_CM) return collide_cm<R, FORCED>(P, s, Fx, Fy);
    R drho = R(0), jx = R(0), jy = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        drho += s[i];
        jx += R(ex(i)) * s[i];
        jy += R(ey(i)) * s[i];
    }
    const R rho = R(1) + drho;
    if (kind == COL_NONE) return rho;
    if (!FORCED && (kind == COL_BGK || kind == COL_TRT)) {
        // Unforced BGK/TRT in a factored form of Eq. 2 (same quantities, fewer
        // operations): with j = rho u and c0 = drho - 1.5 j.u,
        //   seq_i = w_i (c0 + (e_i.j)(3 + 4.5 e_i.u)),
        // and each opposite pair shares e.u and e.j up to sign.
        const R inv = R(1) / rho;
        const R ux = jx * inv, uy = jy * inv;
        const R c0 = drho - R(1.5) * (jx * ux + jy * uy);
        // pairs (i, opp i): e = (1,0), (0,1), (1,1), (-1,1)
        const R eu[4] = {ux, uy, ux + uy, uy - ux};
        const R ej[4] = {jx, jy, jx + jy, jy - jx};
        const int pi[4] = {1, 2, 5, 6}, po[4] = {3, 4, 7, 8};
        if (kind == COL_BGK) {
            const R om = P.omega, oms = R(1) - om;
            s[0] = oms * s[0] + (om * wgt<R>(0)) * c0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const R a = om * wgt<R>(pi[p]);
                const R qp = c0 + ej[p] * (R(3) + R(4.5) * eu[p]);
                const R qm = c0 - ej[p] * (R(3) - R(4.5) * eu[p]);
                s[pi[p]] = oms * s[pi[p]] + a * qp;
                s[po[p]] = oms * s[po[p]] + a * qm;
            }
            return rho;
        }
        // TRT: symmetric part e+ = w (c0 + 4.5 (e.j)(e.u)), antisymmetric e- = 3 w (e.j)
        const R se = P.s_e, so = P.s_o;
        s[0] = s[0] - se * (s[0] - wgt<R>(0) * c0);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const R w = wgt<R>(pi[p]);
            const R sp = R(0.5) * (s[pi[p]] + s[po[p]]), sm = R(0.5) * (s[pi[p]] - s[po[p]]);
            const R dp = se * (sp - w * (c0 + R(4.5) * ej[p] * eu[p]));
            const R dm = so * (sm - R(3) * w * ej[p]);
            s[pi[p]] = s[pi[p]] - dp - dm;
            s[po[p]] = s[po[p]] - dp + dm;
        }
        return rho;
    }
    const R inv = R(1) / rho;
    const R ux = (FORCED ? jx + R(0.5) * Fx : jx) * inv, uy = (FORCED ? jy + R(0.5) * Fy : jy) * inv;   // Eq. 4
    const R uu = ux * ux + uy * uy;
    if (kind == COL_BGK) {
        const R pre = R(1) - R(0.5) * P.omega;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if (FORCED)
                s[i] = s[i] - P.omega * (s[i] - seq_i(i, drho, rho, ux, uy, uu)) + pre * guo_i(i, ux, uy, Fx, Fy);
            else
                s[i] = s[i] - P.omega * (s[i] - seq_i(i, drho, rho, ux, uy, uu));
        }
        return rho;
    }
    if (kind == COL_TRT) {
        const R pe = R(1) - R(0.5) * P.s_e, po = R(1) - R(0.5) * P.s_o;
        R out[9];
        {
            R q = seq_i(0, drho, rho, ux, uy, uu);
            out[0] = s[0] - P.s_e * (s[0] - q);
            if (FORCED) out[0] += pe * guo_i(0, ux, uy, Fx, Fy);
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const int o = opp(i);
            R qi = seq_i(i, drho, rho, ux, uy, uu), qo = seq_i(o, drho, rho, ux, uy, uu);
            R sp = R(0.5) * (s[i] + s[o]), sm = R(0.5) * (s[i] - s[o]);
            R ep = R(0.5) * (qi + qo), em = R(0.5) * (qi - qo);
            out[i] = s[i] - P.s_e * (sp - ep) - P.s_o * (sm - em);
            if (FORCED) {
                R gi = guo_i(i, ux, uy, Fx, Fy), go = guo_i(o, ux, uy, Fx, Fy);
                R gp = R(0.5) * (gi + go), gm = R(0.5) * (gi - go);
                out[i] += pe * gp + po * gm;
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) s[i] = out[i];
        return rho;
    }
    return rho;
}


// ---- domain conditions (Sec. 2.9) -------------------------------------------------------
// Zou-He velocity closure written once for any side from its inward normal n and
// tangent t: rho = (1 + sum_{e.n=0} s + 2 sum_{e.n<0} s) / (1 - u.n) and for every
// unknown population (e.n > 0):
//   s_i = s_opp + 6 w_i rho (e_i.u) + (e_i.t)/2 [ (2/3) rho (u.t) - sum_{e.n=0} s_j (e_j.t) ].
// With ``bounce`` (wall_closure = 1 on a side whose prescribed velocity is exactly zero,
// decided on the host in FP64) the side closes by on-node bounce-back of the unknowns,
// s_i = s_opp: the closure above at u = 0 without its tangential correction.
template <class R>
__device__ __forceinline__ void zou_he(int side, R (&s)[9], R ux, R uy, bool bounce = false) {
    const int nnx = side == SIDE_W ? 1 : (side == SIDE_E ? -1 : 0);
    const int nny = side == SIDE_S ? 1 : (side == SIDE_N ? -1 : 0);
    const int ttx = nnx == 0 ? 1 : 0, tty = nnx == 0 ? 0 : 1;
    if (bounce) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if (ex(i) * nnx + ey(i) * nny > 0) s[i] = s[opp(i)];
        return;
    }
    R a = R(0), b = R(0), Qt = R(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int en = ex(i) * nnx + ey(i) * nny;
        if (en == 0) { a += s[i]; Qt += R(ex(i) * ttx + ey(i) * tty) * s[i]; }
        if (en < 0) b += s[i];
    }
    const R un = ux * R(nnx) + uy * R(nny), ut = ux * R(ttx) + uy * R(tty);
    const R rho = (R(1) + a + R(2) * b) / (R(1) - un);
    const R tr = (R(2) / R(3)) * rho * ut - Qt;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int en = ex(i) * nnx + ey(i) * nny;
        if (en > 0) {
            const R eu = R(ex(i)) * ux + R(ey(i)) * uy;
            const int et = ex(i) * ttx + ey(i) * tty;
            s[i] = s[opp(i)] + R(6) * wgt<R>(i) * rho * eu + R(0.5) * R(et) * tr;
        }
    }
}

// Pure streaming pull of the nine populations arriving at (x, y); sources
// outside a non-periodic lattice give 0 (unknowns, set by a domain condition).
template <class S, class R>
__device__ __forceinline__ void pull_node(const CaseDev& C, const S* __restrict__ src, int x, int y, R (&s)[9]) {
    const bool xper = C.bc[SIDE_W] == BC_PER, yper = C.bc[SIDE_S] == BC_PER;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - ex(i), sy = y - ey(i);
        if (xper) sx = sx < 0 ? sx + C.nx : (sx >= C.nx ? sx - C.nx : sx);
        if (yper) sy = sy < 0 ? sy + C.ny : (sy >= C.ny ? sy - C.ny : sy);
        const bool in = sx >= 0 && sx < C.nx && sy >= 0 && sy < C.ny;
        s[i] = in ? ld1(src + i * C.plane + (long long)sy * C.pitch + sx) : R(0);
    }
}

// Post-streaming populations at (x, y) with the domain conditions applied:
// edges use Zou-He or the zero-gradient copy of the adjacent interior node;
// corners copy the diagonal interior node (both sides zero-gradient) or take
// the equilibrium at its density and the prescribed velocity (mean of both
// sides when both prescribe one).
template <class S, class R>
__device__ void post_stream_node(const CaseDev& C, const S* __restrict__ src, int x, int y, R (&s)[9]) {
    const bool xper = C.bc[SIDE_W] == BC_PER, yper = C.bc[SIDE_S] == BC_PER;
    const bool xw = !xper && x == 0, xe = !xper && x == C.nx - 1;
    const bool ys = !yper && y == 0, yn = !yper && y == C.ny - 1;
    if (!(xw || xe || ys || yn)) { pull_node<S, R>(C, src, x, y, s); return; }
    if ((xw || xe) && (ys || yn)) {
        const int sx = xw ? SIDE_W : SIDE_E, sy = ys ? SIDE_S : SIDE_N;
        R d[9];
        pull_node<S, R>(C, src, xw ? 1 : C.nx - 2, ys ? 1 : C.ny - 2, d);
        if (C.bc[sx] == BC_NEU && C.bc[sy] == BC_NEU) {
#pragma unroll
            for (int i = 0; i < 9; ++i) s[i] = d[i];
            return;
        }
        R drho = R(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) drho += d[i];
        double ux, uy;
        if (C.bc[sx] == BC_VEL && C.bc[sy] == BC_VEL) {
            ux = 0.5 * (C.ubc[sx][0] + C.ubc[sy][0]);
            uy = 0.5 * (C.ubc[sx][1] + C.ubc[sy][1]);
        } else if (C.bc[sx] == BC_VEL) {
            ux = C.ubc[sx][0]; uy = C.ubc[sx][1];
        } else {
            ux = C.ubc[sy][0]; uy = C.ubc[sy][1];
        }
        const R rux = R(ux), ruy = R(uy), uu = rux * rux + ruy * ruy;
#pragma unroll
        for (int i = 0; i < 9; ++i) s[i] = seq_i(i, drho, R(1) + drho, rux, ruy, uu);
        return;
    }
    const int side = xw ? SIDE_W : (xe ? SIDE_E : (ys ? SIDE_S : SIDE_N));
    if (C.bc[side] == BC_NEU) {
        const int ix = xw ? 1 : (xe ? C.nx - 2 : x), iy = ys ? 1 : (yn ? C.ny - 2 : y);
        pull_node<S, R>(C, src, ix, iy, s);
        return;
    }
    pull_node<S, R>(C, src, x, y, s);
    zou_he<R>(side, s, R(C.ubc[side][0]), R(C.ubc[side][1]), (C.wall_bb >> side) & 1);
}

// ---- regularised delta kernels (Eq. 9, Eq. 10) --------------------------------------------
template <class R>
__device__ __forceinline__ R phi(int kernel, R r) {
    const R a = fabs(r);
    if (kernel == K_HAT) return a < R(1) ? R(1) - a : R(0);
    if (a <= R(1)) return (R(3) - R(2) * a + sqrt(R(1) + R(4) * a - R(4) * a * a)) / R(8);
    if (a <= R(2)) return (R(5) - R(2) * a - sqrt(R(-7) + R(12) * a - R(4) * a * a)) / R(8);
    return R(0);
}

}  // namespace iblbm
