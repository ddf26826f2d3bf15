// lbm_internal.cuh -- device-side types of the GB300 LBM / moving-particle
// library.  Lattice Boltzmann method with fully resolved rigid particles,
// Sec. 4 of Bartuschat et al. ("Two computational models for simulating the
// tumbling motion of elongated particles in fluids").
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include "../../include/lbm.h"

namespace lbm {

constexpr int Q = 19;

// D3Q19 (Sec. 4.1).  Numbering: 0 rest, 1..6 axis pairs, 7..18 diagonal pairs;
// q and opp(q) are adjacent so opp is arithmetic.  Indexed only with
// compile-time q (unrolled loops), so the tables fold into immediates.
__host__ __device__ constexpr int cx(int q) {
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int cy(int q) {
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int cz(int q) {
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr double wq(int q) {
    return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Internal cell flags (one byte per cell).
constexpr uint8_t F_NEAR = 1;     // fluid cell with at least one wall/obstacle neighbour
constexpr uint8_t F_SOLID = 2;    // wall or obstacle cell (not collided)
constexpr uint8_t F_CHANGED = 4;  // touched by this step's re-mapping (transient)
constexpr uint8_t F_WALL = 8;     // static wall layer (never re-mapped)
// Fluid cells (with F_NEAR) whose wall/obstacle neighbours all belong to the
// moving wall layer y = 0 (F_YLO) or y = ny-1 (F_YHI) of a non-periodic y
// axis: their bounced directions are exactly those with c_y = -1 (resp. +1).
// wall cell whose wall-layer axes are all free-slip: a link into it reflects
// instead of bouncing back, and the odd step pulls through it like a fluid cell
constexpr uint8_t F_FSLIP = 64;
constexpr uint8_t F_YLO = 16;
constexpr uint8_t F_YHI = 32;

constexpr uint32_t PID_FLUID = LBM_PID_FLUID;
constexpr uint32_t PID_WALL_YLO = LBM_PID_WALL_YLO;
constexpr uint32_t PID_WALL_YHI = LBM_PID_WALL_YHI;
constexpr uint32_t PID_WALL = LBM_PID_WALL;

// Division by a runtime-invariant divisor with one multiply-high
// (Granlund & Montgomery, PLDI 1994, round-up variant): exact for n < 2^31.
struct FastDiv {
    uint32_t d, m, s;
    __host__ void init(uint32_t div) {
        d = div;
        s = 0;
        while ((1ull << s) < div) ++s;
        m = (uint32_t)((((1ull << 32) * ((1ull << s) - div)) / div) + 1);
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        return (__umulhi(n, m) + n) >> s;
    }
};

// One lattice of a context (device-resident table, one entry per lattice).
struct LatDev {
    int nx, ny, nz;
    int n;                 // nx*ny*nz
    int npad;              // population plane stride (elements)
    int tile0;             // first sweep tile of this lattice
    long long f_off;       // element offset of plane 0 in the population arena
    long long c_off;       // cell offset in the flag / id arenas
    FastDiv divx, divxy;   // idx -> (x, y, z)
    int px, py, pz;        // periodic flags
    int fsx, fsy, fsz;     // free-slip wall layers (non-periodic axes only)
    double omega, omega_odd, rho0;
    double inv_rho0;       // 1 / rho0
    double rho18;          // rho0 / 18: 2 w_q rho0 = (36 w_q) rho0 / 18 with 36 w_q in {1, 2}
    double wlo[3], whi[3], g[3];
    float rho18f[2];       // rho0 / 18 as a double-float (hi, lo)
    // FP32 copies of the relaxation and boundary parameters: a double -> float
    // conversion issues on GB300's narrow FP64 pipe, so the FP32/FP16/BF16
    // sweeps read these instead of converting per cell
    float fomega, fomega_odd, frho0, finv_rho0;
    float fg[3], fwlo[3], fwhi[3];
    // learned closure scales: shear rate of the channel between the moving
    // y walls (0 without them: no closure) and dynamic viscosity
    float cl_gamma, cl_mu;
    int off[Q];            // linear offset of x + c_q for cells off the periodic faces
    // TRT collision constants (Eqs. TRTOp, EqPDF_TRT regrouped, see collide):
    // kd / kf = {1 - om, om w_0, -1.5 rho0, (1 - om)/2, (1 - oo)/2, om w_1,
    // om w_2, 4.5 rho0 om w_1, 4.5 rho0 om w_2, 3 rho0 oo w_1, 3 rho0 oo w_2}
    // (w_1 = 1/18 axis, w_2 = 1/36 diagonal directions), and per direction
    // pair i (q = 2i + 1) the body-force source 3 w_q rho0 c_q.g
    double kd[11], fsd[9];
    float kf[11], fsf[9];
    // momentum stabilisation (Sec. 4.1): mean fluid velocity of the current
    // step, subtracted from u in every equilibrium; null when off
    const double *ubar;
    const float *ubarf;
};

// Lattice parameters in the compute precision C (FP64 fields for double, the
// FP32 copies otherwise).
template <class C> struct LatPar {
    C omega, omega_odd, rho0, inv_rho0, g[3], wlo[3], whi[3], ubar[3];
    __device__ __forceinline__ explicit LatPar(const LatDev &L) {
        if constexpr (sizeof(C) == 8) {
            omega = L.omega; omega_odd = L.omega_odd; rho0 = L.rho0; inv_rho0 = L.inv_rho0;
            for (int k = 0; k < 3; ++k) { g[k] = L.g[k]; wlo[k] = L.wlo[k]; whi[k] = L.whi[k]; }
            for (int k = 0; k < 3; ++k) ubar[k] = L.ubar ? L.ubar[k] : 0.0;
        } else {
            omega = L.fomega; omega_odd = L.fomega_odd; rho0 = L.frho0; inv_rho0 = L.finv_rho0;
            for (int k = 0; k < 3; ++k) { g[k] = L.fg[k]; wlo[k] = L.fwlo[k]; whi[k] = L.fwhi[k]; }
            for (int k = 0; k < 3; ++k) ubar[k] = L.ubarf ? L.ubarf[k] : 0.0f;
        }
    }
};

// Rigid bodies, structure of arrays, FP64 throughout.
struct PartDev {
    int np;
    int pad0;
    double *pos, *quat, *vel, *om, *L;   // current state (3/4/3/3/3 per body)
    double *semi, *mass, *inertia;       // shape: semi-axes, mass, body inertia diag
    double *minv, *Iinv;                 // 1/mass, 1/inertia (host-computed)
    float *bodyf;                        // BF_STRIDE per body, layout BF_* below
    double *R64;                         // 9 per body: rotation of quat, rounded as the mapping's inside test
    float *feat;                         // learned closure: features, CL_IN per body
    double *extF, *extM;                 // external loads
    int *cell, *fixed;
    double *pos_old, *vel_old, *om_old, *quat_old; // state before this step's update
    double *acc;       // 6 per body: hydrodynamic F, M summed by the sweep
    double *last;      // 6 per body: F, M of the last completed step
    int *region;       // 6 per body: lo[3], ext[3] of the re-mapping box
    int *changed;      // per body: this step's uncover / claim changed a cell's owner (fix-up and flags run)
};

// FP32 copy of a body's pose and motion (PartDev::bodyf, BF_STRIDE floats per
// body): rotation matrix, reciprocal semi-axes, centre as a double-float
// (hi at BF_POS, lo at BF_POSLO), translational and angular velocity, the
// shape (BF_SHAPE: 0 ellipsoid, 1 spherocylinder) and, for a spherocylinder
// of radius r and half length a, the half length of its cylindrical part in
// units of r, (a - r) / r (BF_CAPH; 0 for an ellipsoid).  BF_TUBE_H and
// BF_TUBE_R: half length and radius of the cylinder about the body x axis
// that holds every cell the re-mapping passes can touch this step (the body's
// own cylinder, semi_0 and max(semi_1, semi_2), widened by the step's largest
// displacement of a body point and a margin of two cells).
constexpr int BF_STRIDE = 32;
constexpr int BF_R = 0, BF_INV = 9, BF_POS = 12, BF_POSLO = 16, BF_U = 19, BF_W = 22, BF_CAPH = 25,
              BF_SHAPE = 26, BF_TUBE_H = 27, BF_TUBE_R = 28;

struct SweepArgs {
    LatDev lat0;             // copy of lattice 0 (used when nlat == 1)
    const LatDev *lat;
    int nlat;
    int ntiles;
    void *f;                 // population arena (storage type)
    const uint8_t *flags;
    const uint32_t *pid;
    PartDev P;
    double *wall_acc;        // 6 per lattice: y-low wall F, y-high wall F
    uint32_t *err;           // device error word
    // direct sweep: bit t of tbits set = tile t may hold a cell with a nonzero
    // flag; a clear bit guarantees that every cell of the tile is bulk fluid
    // (null: every tile is treated as flagged)
    const uint32_t *tbits;
    const uint64_t *links;   // per cell: neighbour masks (LK_* layout)
    const uint32_t *nbody;   // per cell: first body among the neighbours
    // split direct sweep (null: near cells stay in the sweep): the sweep skips
    // near-obstacle cells, a list kernel compacts them into near_list
    // (global cell indices, *near_count of them) and a second kernel
    // updates them with every lane busy
    uint32_t *near_list;
    uint32_t *near_count;
    const int *tile_lat;     // batches: lattice of every tile (null: binary search on tile0)
    const uint32_t *tick;    // step counter (seed of the BF16 stochastic rounding)
    // direct sweep: a block starting tile t asks the L2 to fetch the
    // population ranges of tile t + pf_ahead[parity] (0: no prefetch), per
    // step parity (index 0: even-step sweeps, 1: odd)
    int pf_ahead[2];
};

// Stochastic rounding of the BF16 sweep stores.  A bfloat16 keeps 8
// significant bits; rounded to nearest, a population that changes little from
// step to step gets the same rounding error every step, and on flows that are
// uniform along whole planes (shear between walls) that error is the same over
// the plane, a steady bias that the flow integrates.  The sweep's BF16 stores
// therefore round up with probability equal to the discarded fraction of the
// FP32 value (unbiased), driven by a counter-based generator: a per-step seed
// from the context's step counter (advanced by the rigid-body kernel), hashed
// with the cell index by Wellons' "lowbias32" integer hash, then one step of
// the Numerical Recipes linear congruential generator per stored population,
// whose upper 16 bits are the rounding bits.  Deterministic for a given state
// and step; FP16, FP32 and FP64 stores round to nearest even.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// Per-step seed from the step counter (null: 0).
__device__ __forceinline__ uint32_t step_seed(const uint32_t *tick) {
    return tick ? mix32(*tick * 0x9e3779b9u + 0x632be5abu) : 0u;
}
template <int PREC> struct Rnd {
    __device__ __forceinline__ Rnd(uint32_t, long long) {}
    __device__ __forceinline__ uint32_t next() { return 0u; }
};
template <> struct Rnd<LBM_BF16_OFFSET> {
    uint32_t s;
    __device__ __forceinline__ Rnd(uint32_t seed, long long cell) : s(mix32(seed ^ (uint32_t)cell)) {}
    __device__ __forceinline__ uint32_t next() {
        s = s * 1664525u + 1013904223u;
        return s >> 16;
    }
};
// FP32 -> BF16 bits, rounded up with probability (discarded bits) / 2^16 for
// r16 uniform in [0, 2^16): adding r16 below the kept 16 bits and truncating
// (a carry into the exponent is the correct next value); non-finite values
// convert as rounding to nearest does.
__device__ __forceinline__ unsigned short bf16_bits_sr(float v, uint32_t r16) {
    const uint32_t b = __float_as_uint(v);
    if ((b & 0x7f800000u) == 0x7f800000u) return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    return (unsigned short)((b + r16) >> 16);
}

// Storage forms: every form holds g_q = f_q - w_q rho0 (the offset from rest).
// ld / st work on any address space (global, shared stage, local); ldg / stg
// are for populations in global memory only: the sweep touches each once per
// step and the arrays are larger than L2, so they carry the streaming
// (evict-first) cache hint, ld.global.cs / st.global.cs (measured 4-5 %
// faster sweeps on GB300).  A .global access on a shared or local address is
// an invalid-address-space fault, so stage and register copies use ld / st.
// stg(p, v, r16) is the sweep's store: r16 are the rounding bits of Rnd (used
// by the BF16 form only).  bits(v, r16) gives the stored bit pattern.
template <int PREC> struct Store;
template <> struct Store<LBM_F64> {
    using T = double;
    using C = double;
    static __device__ __forceinline__ C ld(const T *p) { return *p; }
    static __device__ __forceinline__ void st(T *p, C v) { *p = v; }
    static __device__ __forceinline__ C ldg(const T *p) { return __ldcs(p); }
    static __device__ __forceinline__ void stg(T *p, C v) { __stcs(p, v); }
    static __device__ __forceinline__ void stg(T *p, C v, uint32_t) { __stcs(p, v); }
};
template <> struct Store<LBM_F32> {
    using T = float;
    using C = float;
    static __device__ __forceinline__ C ld(const T *p) { return *p; }
    static __device__ __forceinline__ void st(T *p, C v) { *p = v; }
    static __device__ __forceinline__ C ldg(const T *p) { return __ldcs(p); }
    static __device__ __forceinline__ void stg(T *p, C v) { __stcs(p, v); }
    static __device__ __forceinline__ void stg(T *p, C v, uint32_t) { __stcs(p, v); }
};
template <> struct Store<LBM_F16_OFFSET> {
    using T = __half;
    using C = float;
    static __device__ __forceinline__ C ld(const T *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(T *p, C v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ C ldg(const T *p) { return __half2float(__ldcs(p)); }
    static __device__ __forceinline__ void stg(T *p, C v) { __stcs(p, __float2half_rn(v)); }
    static __device__ __forceinline__ void stg(T *p, C v, uint32_t) { __stcs(p, __float2half_rn(v)); }
    static __device__ __forceinline__ unsigned short bits(C v, uint32_t) {
        return __half_as_ushort(__float2half_rn(v));
    }
    static __device__ __forceinline__ C from_bits(unsigned short h) { return __half2float(__ushort_as_half(h)); }
};
template <> struct Store<LBM_BF16_OFFSET> {
    using T = __nv_bfloat16;
    using C = float;
    static __device__ __forceinline__ C ld(const T *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(T *p, C v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ C ldg(const T *p) { return __bfloat162float(__ldcs(p)); }
    static __device__ __forceinline__ void stg(T *p, C v) { __stcs(p, __float2bfloat16_rn(v)); }
    static __device__ __forceinline__ void stg(T *p, C v, uint32_t r16) {
        __stcs(reinterpret_cast<unsigned short *>(p), bf16_bits_sr(v, r16));
    }
    static __device__ __forceinline__ unsigned short bits(C v, uint32_t r16) { return bf16_bits_sr(v, r16); }
    static __device__ __forceinline__ C from_bits(unsigned short h) {
        return __bfloat162float(__ushort_as_bfloat16(h));
    }
};


// Force/torque accumulators are kept in ACC_COPIES copies per body (and per
// lattice wall pair); a warp adds into copy (8*block + warp) mod ACC_COPIES,
// which spreads same-address FP64 atomics, and the rigid-body kernel sums the
// copies.  Layout: body p, copy c -> acc[(p*ACC_COPIES + c)*6 + k] (F then M);
// lattice l, copy c -> wall_acc[(l*ACC_COPIES + c)*6 + 3*side + k].
constexpr int ACC_COPIES = 32;

// Double-float numbers: the unevaluated sum hi + lo of two FP32 values
// (about 48 significant bits), built from error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2) and the FMA product error
// (Ogita, Rump & Oishi 2005), renormalised as in Bailey's double-double
// addition.  Every operation is an explicitly rounded FP32 intrinsic, so the
// compiler neither contracts nor reorders them.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s = two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df df_add_f(df a, float b) {
    const df s = two_sum(a.hi, b);
    return two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    return two_sum(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}
__device__ __forceinline__ df df_from_double(double x) {
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// Programmatic dependent launch.  The kernels of a time step form one
// dependent chain (sweep, rigid bodies, re-mapping passes, next sweep); each is
// launched with programmatic stream serialisation, so it can be scheduled
// while its predecessor is still running.  Every such kernel calls pdl_wait()
// before it touches global memory (it returns once the predecessor grid has
// completed and its writes are visible) and then pdl_trigger(), which lets
// the successor be scheduled as soon as all of this grid's blocks have
// started.  Without a programmatic predecessor pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Device error-word bits.
constexpr uint32_t ERR_NONFINITE = 1u;
constexpr uint32_t ERR_TIMEOUT = 2u;
constexpr uint32_t ERR_FSLIP_BODY = 4u;  // a body reached the fluid layer next to a free-slip wall

// --- launchers (defined in the .cu files) ---------------------------------
// Sweep variants: direct (`cpt` consecutive cells per thread, `block`
// threads per block, tiles of cpt * block cells), staged (tiles of 256 cells
// brought into shared memory by bulk asynchronous copies) and ring
// (per-thread asynchronous prefetch ring, block 256).
constexpr int SWEEP_DIRECT = 0;
constexpr int SWEEP_STAGED = 1;
constexpr int SWEEP_RING = 2;
cudaError_t launch_sweep(int prec, int parity, int variant, const SweepArgs &a, int grid, int block, int cpt,
                         cudaStream_t s);
template <int PREC>
cudaError_t launch_sweep_prec(int parity, int variant, const SweepArgs &a, int grid, int block, int cpt,
                              cudaStream_t s);
template <int PREC> int sweep_max_blocks_prec(int variant, int block, int cpt);
// Cells per thread the direct sweep supports in storage form prec (1, 2, 4).
inline bool sweep_cpt_supported(int prec, int cpt) {
    return cpt == 1 || cpt == 2 || (cpt == 4 && prec != LBM_F64);
}
// Fill map[t] = lattice of tile t for the current tile size (lat: device table).
cudaError_t launch_tile_map(const LatDev *lat, int nlat, int ntiles, int *map, cudaStream_t s);

// Learned closure (see lbm_closure.cu): features of every body, network
// inference (applied to the bodies' accumulators, or written out), training.
constexpr int CL_IN = 86, CL_HID = 64, CL_OUT = 6, CL_PARAMS = 14278;
struct ClosureArgs {
    const LatDev *lat;
    const void *f;
    const uint8_t *flags;
    PartDev P;
    float *feat;  // CL_IN per body
};
struct MlpArgs {
    __half *par16;        // FP16 working parameters (CL_PARAMS)
    float *par32;         // FP32 master parameters (training)
    float *adam_m, *adam_v;
    float *grad;          // CL_PARAMS
    const float *x;       // n x CL_IN
    const float *y;       // n x CL_OUT targets (training)
    float *out;           // n x CL_OUT outputs (inference without apply)
    float *loss;          // device scalar (may be null)
    int n;
};
cudaError_t launch_closure_features(int prec, int next_odd, const ClosureArgs &a, cudaStream_t s);
cudaError_t launch_mlp_infer(const MlpArgs &m, const ClosureArgs *apply, cudaStream_t s);
cudaError_t launch_mlp_grad(const MlpArgs &m, cudaStream_t s);
cudaError_t launch_adam(const MlpArgs &m, float lr, float beta1, float beta2, float eps, float c1, float c2,
                        cudaStream_t s);
cudaError_t launch_to_half(const float *src, __half *dst, int n, cudaStream_t s);
int sweep_max_active_blocks(int prec, int variant, int block, int cpt);
constexpr int STAGED_TILE = 256;

// Link word of a fluid cell (PartDev-independent, kept by the flags pass):
// bit q (1..18) of each 19-bit field refers to the neighbour x + c_q --
// field 0: wall or obstacle cell, field 1: wall-layer cell, field 2: cell of
// the first body met in q order (whose id is kept in nbody).  Zero for cells
// without wall or obstacle neighbours and for solid cells.
constexpr int LK_WALL = 19, LK_BODY = 38;
constexpr uint32_t LK_MASK = 0x7FFFFu;

struct RemapArgs {
    const LatDev *lat;
    void *f;
    uint8_t *flags;
    uint32_t *pid;
    uint32_t *pid_prev;
    PartDev P;
    double *wall_acc;
    double *wall_last;
    int nlat;
    uint32_t *err;
    uint32_t *tbits;     // direct-sweep tile bits (may be null)
    int tile;            // cells per direct-sweep tile
    uint64_t *links;     // per-cell link words (LK_* layout)
    uint32_t *nbody;     // per-cell first neighbouring body
    uint32_t *tick;      // step counter, advanced once per rigid-body update
    // cells whose owner changed in this step's uncover / claim passes, each
    // listed once (the pass that sets its F_CHANGED bit lists it); the
    // rigid-body update empties the list.  chg_cap: the arena's cell count
    uint32_t *chg;
    uint32_t *chg_n;
    long long chg_cap;
};
// Recount every tile bit from the flags (bit t = tile t holds a nonzero flag).
cudaError_t launch_tile_bits(const RemapArgs &a, int ntiles, cudaStream_t s);
cudaError_t launch_rigid_body(const RemapArgs &a, cudaStream_t s);
cudaError_t launch_remap_step(int prec, int next_parity, const RemapArgs &a, int blocks_per_body,
                              cudaStream_t s);
// Fused re-mapping step (rigid-body update and the four region passes in one
// cooperative launch with grid barriers).  GridBar: zero-initialised device
// state of the barrier, left at count 0 by every completed launch.
struct GridBar {
    unsigned count, gen;
    unsigned limit;  // polls before a wait gives up (0: the default, 2^20)
};
// Co-resident blocks of the fused kernel over the device (0: no cooperative launch).
int remap_fused_max_blocks();
// Launch form the device and driver accept eagerly and in a captured graph:
// 2 cooperative with a programmatic dependency, 1 cooperative, 0 none.
int remap_fused_probe();
cudaError_t launch_remap_fused(int prec, int next_parity, const RemapArgs &a, int blocks_per_body, int grid,
                               int mode, GridBar *bar, cudaStream_t s);
// Momentum stabilisation (Sec. 4.1) of a single lattice: sum the
// pre-collision velocity j / rho0 and the count of fluid cells into acc[0..3]
// (the state the sweep of parity next_parity reads), then turn the sums into
// the mean velocity (acc[4..6], FP32 copy in accf[0..2]) and clear them.
cudaError_t launch_momentum_mean(int prec, int next_parity, const LatDev &h, const LatDev *d, const void *f,
                                 const uint8_t *flags, double *acc, float *accf, cudaStream_t s);
cudaError_t launch_clear_particles(const LatDev &h, const RemapArgs &a, int lat_index,
                                   cudaStream_t s);
cudaError_t launch_claim_all(const RemapArgs &a, int blocks_per_body, cudaStream_t s);
cudaError_t launch_remap_full(int prec, int next_parity, const RemapArgs &a, const LatDev &h,
                              int lat_index, cudaStream_t s);
cudaError_t launch_init_cells(const LatDev &h, const LatDev *d, uint8_t *flags, uint32_t *pid,
                              uint32_t *pid_prev, uint64_t *links, uint32_t *nbody, cudaStream_t s);
cudaError_t launch_canonical(int prec, int next_parity, const LatDev &h, const LatDev *d,
                             const void *f, const uint8_t *flags, const uint32_t *pid,
                             double *rho, double *u3, uint8_t *flags_out, double *pdfs,
                             cudaStream_t s);
cudaError_t launch_set_pdfs(int prec, int next_parity, const LatDev &h, const LatDev *d, void *f,
                            const uint8_t *flags, const double *pdfs, cudaStream_t s);
cudaError_t launch_links(const LatDev &h, const LatDev *d, const uint8_t *flags,
                         const uint32_t *pid, int *block_counts, int nblocks, int32_t *idx,
                         int8_t *q, uint32_t *pid_out, int cap, int *total, cudaStream_t s);
int kernels_per_remap_step(int np);

}  // namespace lbm
