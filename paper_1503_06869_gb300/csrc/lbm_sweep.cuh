// lbm_sweep.cuh -- the fused stream-collide sweep (Sec. 4.1, Eqs. LBMCollide and
// LBMStream, with the boundary treatment folded into the sweep as in Sec. 4.4)
// for D3Q19 TRT with the incompressible equilibrium (Eqs. fequ_Incompr,
// TRTOp, EqPDF_TRT), velocity bounce-back at walls and moving obstacle cells
// (Eqs. BBBC, LBMMovWall) and the momentum-exchange force and torque per
// particle (Eqs. TransferredMomentum, LBMhydrodynForce).
//
// Memory layout: populations of a lattice are structure-of-arrays planes
// g[q][idx] (idx = x + nx(y + ny z), x fastest), one buffer, updated in place
// with the AA pattern (Bailey et al. 2009):
//   even step: read slot q of x, write the post-collision value of q to slot
//              opp(q) of x  -- no neighbour access at all;
//   odd step:  read slot opp(p) of x - c_p, write slot q of x + c_q.
// Each memory slot is read and then written by the same thread, so the sweep
// needs no second buffer and no synchronisation.  Bounce-back is applied when
// a value is written: a value leaving x towards an obstacle (x + c_q solid)
// becomes f~_q - 6 w_q rho0 c_q.u_s and is written to the slot from which the
// next step reads f_opp(q)(x): slot opp(q) of x in both parities.  On odd
// steps the read of f_p(x) comes from slot p of x itself when x - c_p is an
// obstacle (that is where the previous even step put the bounced value).
//
// Fluid cells without obstacle neighbours (flag 0) take a branch with no
// flag or id reads beyond their own flag byte; only cells flagged F_NEAR read
// neighbour flags, obstacle ids and particle state.
//
// Included once per storage form by lbm_sweep_<form>.cu, each of which
// instantiates launch_sweep_prec / sweep_max_blocks_prec for its form (the
// forms compile in parallel); lbm_sweep.cu dispatches on the form.
#pragma once
#include <mutex>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr uint32_t SLOT_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t KEY_WALL = 0x80000000u;

// Lattice tables for runtime-indexed use in the bounce-back helper.
__constant__ int c_cx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int c_cy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int c_cz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
// direction index of (cx, cy, cz) at (cx + 1) + 3 (cy + 1) + 9 (cz + 1); -1: none
__constant__ int c_qidx[27] = {-1, 16, -1, 12, 6, 13, -1, 17, -1, 8, 4, 9, 2, 0, 1, 10, 3, 7,
                               -1, 18, -1, 14, 5, 11, -1, 15, -1};
__constant__ double c_w[Q] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0};

__device__ __forceinline__ double *global_acc(const SweepArgs &a, uint32_t key) {
    const size_t c = (blockIdx.x * 8u + (threadIdx.x >> 5)) & (ACC_COPIES - 1);
    if (key & KEY_WALL) {
        const size_t l = (key & ~KEY_WALL) >> 1;
        return a.wall_acc + 6 * (l * ACC_COPIES + c) + 3 * (key & 1u);
    }
    return a.P.acc + 6 * ((size_t)key * ACC_COPIES + c);
}

__device__ __forceinline__ double min_image(double d, int n, int periodic) {
    if (periodic) {
        if (d > 0.5 * n)
            d -= n;
        else if (d < -0.5 * n)
            d += n;
    }
    return d;
}

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// TRT collision in offset form, in place: on entry g holds f - w rho0, on
// exit the post-collision offsets f~ - w rho0.  With dr = sum g = rho - rho0
// the even equilibrium offset is w (dr - 1.5 rho0 u.u + 4.5 rho0 (c.u)^2),
// the odd one 3 w rho0 c.u (Eq. EqPDF_TRT with c_s^2 = 1/3); the body force
// enters as the odd source 3 w rho0 c.g.  Under momentum stabilisation
// (Sec. 4.1) the equilibria are taken at u - ubar (ubar = 0 otherwise).
// Evaluated per direction pair (q, opp(q)) from the pair sum s = f_q +
// f_opp(q) and difference d = f_q - f_opp(q), which also give the moments.
// With the even and odd parts s/2, d/2 (Eq. TRTOp) and e = w base + 4.5 w
// rho0 (c.u)^2, o = 3 w rho0 (c.u) + 3 w rho0 c.g the update
// f~_q = f_q - om (s/2 - e) - (oo (d/2 - o') ...) regroups to
//   f~_q = [(1 - om)/2 s + om e] + [(1 - oo)/2 d + oo 3 w rho0 c.u + 3 w rho0 c.g],
//   f~_opp(q) = [first bracket] - [second bracket],
// (o' the odd equilibrium without the source, which enters unrelaxed) so a
// pair costs about seven fused operations; the products of the relaxation
// rates, weights and rho0 are per-lattice constants k, and fs_i = 3 w rho0 c.g.
template <class C>
__device__ __forceinline__ void collide(C (&g)[Q], const C (&k)[11], const C (&fs)[9], C inv, C bx, C by, C bz) {
    C s[9], d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        s[i] = g[2 * i + 1] + g[2 * i + 2];
        d[i] = g[2 * i + 1] - g[2 * i + 2];
    }
    const C dr = g[0] + (((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + s[8]);
    C jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int q = 2 * i + 1;
        if (cx(q)) jx += cx(q) > 0 ? d[i] : -d[i];
        if (cy(q)) jy += cy(q) > 0 ? d[i] : -d[i];
        if (cz(q)) jz += cz(q) > 0 ? d[i] : -d[i];
    }
    const C ux = jx * inv - bx, uy = jy * inv - by, uz = jz * inv - bz;
    const C base = k[2] * (ux * ux + uy * uy + uz * uz) + dr;
    g[0] = k[0] * g[0] + k[1] * base;
    const C e1 = k[5] * base, e2 = k[6] * base;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int q = 2 * i + 1;
        const bool axis = q <= 6;
        C cu = 0;
        if (cx(q)) cu += cx(q) > 0 ? ux : -ux;
        if (cy(q)) cu += cy(q) > 0 ? uy : -uy;
        if (cz(q)) cu += cz(q) > 0 ? uz : -uz;
        const C even = k[3] * s[i] + ((axis ? k[7] : k[8]) * (cu * cu) + (axis ? e1 : e2));
        const C odd = k[4] * d[i] + ((axis ? k[9] : k[10]) * cu + fs[i]);
        g[q] = even + odd;
        g[q + 1] = even - odd;
    }
}

template <class C>
__device__ __forceinline__ void collide_lat(C (&g)[Q], const LatDev &L) {
    if constexpr (sizeof(C) == 8) {
        const double bx = L.ubar ? L.ubar[0] : 0.0, by = L.ubar ? L.ubar[1] : 0.0, bz = L.ubar ? L.ubar[2] : 0.0;
        collide<double>(g, L.kd, L.fsd, L.inv_rho0, bx, by, bz);
    } else {
        const float bx = L.ubarf ? L.ubarf[0] : 0.0f, by = L.ubarf ? L.ubarf[1] : 0.0f,
                    bz = L.ubarf ? L.ubarf[2] : 0.0f;
        collide<float>(g, L.kf, L.fsf, L.finv_rho0, bx, by, bz);
    }
}

// The same collision for two cells at once (x: one cell, y: the next), on
// Blackwell's paired FP32 instructions (one fused multiply-add, add or
// multiply for both cells per issue slot): the grouped sweep's bulk path is
// bound by instruction issue in the 16-bit storage forms, and the collision
// is most of its arithmetic.  Every operation is explicitly rounded, so the
// results agree with the one-cell collision to rounding (the compiler's
// contraction choices there may differ).
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_bc(float a) { return make_float2(a, a); }

__device__ __forceinline__ void collide2(float2 (&g)[Q], const float (&k)[11], const float (&fs)[9], float inv,
                                         float bx, float by, float bz) {
    float2 s[9], d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        s[i] = p_add(g[2 * i + 1], g[2 * i + 2]);
        d[i] = p_sub(g[2 * i + 1], g[2 * i + 2]);
    }
    const float2 dr = p_add(g[0], p_add(p_add(p_add(p_add(s[0], s[1]), p_add(s[2], s[3])),
                                              p_add(p_add(s[4], s[5]), p_add(s[6], s[7]))), s[8]));
    // momentum components: signed sums of the pair differences (the first
    // term of each starts the sum, so no zero is added)
    float2 j[3];
    bool started[3] = {false, false, false};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int q = 2 * i + 1;
        const int c[3] = {cx(q), cy(q), cz(q)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            if (!started[a]) {
                j[a] = c[a] > 0 ? d[i] : make_float2(-d[i].x, -d[i].y);
                started[a] = true;
            } else {
                j[a] = c[a] > 0 ? p_add(j[a], d[i]) : p_sub(j[a], d[i]);
            }
        }
    }
    const float2 ux = p_fma(j[0], p_bc(inv), p_bc(-bx)), uy = p_fma(j[1], p_bc(inv), p_bc(-by)),
                 uz = p_fma(j[2], p_bc(inv), p_bc(-bz));
    const float2 base = p_fma(p_bc(k[2]), p_fma(ux, ux, p_fma(uy, uy, p_mul(uz, uz))), dr);
    g[0] = p_fma(p_bc(k[0]), g[0], p_mul(p_bc(k[1]), base));
    const float2 e1 = p_mul(p_bc(k[5]), base), e2 = p_mul(p_bc(k[6]), base);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int q = 2 * i + 1;
        const bool axis = q <= 6;
        const float2 u[3] = {ux, uy, uz};
        const int c[3] = {cx(q), cy(q), cz(q)};
        float2 cu = make_float2(0.f, 0.f);
        bool first = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!c[a]) continue;
            if (first) {
                cu = c[a] > 0 ? u[a] : make_float2(-u[a].x, -u[a].y);
                first = false;
            } else {
                cu = c[a] > 0 ? p_add(cu, u[a]) : p_sub(cu, u[a]);
            }
        }
        const float2 even = p_fma(p_bc(k[3]), s[i], p_fma(p_bc(axis ? k[7] : k[8]), p_mul(cu, cu), axis ? e1 : e2));
        const float2 odd = p_fma(p_bc(k[4]), d[i], p_fma(p_bc(axis ? k[9] : k[10]), cu, p_bc(fs[i])));
        g[q] = p_add(even, odd);
        g[q + 1] = p_sub(even, odd);
    }
}

__device__ __forceinline__ void collide2_lat(float2 (&g)[Q], const LatDev &L) {
    const float bx = L.ubarf ? L.ubarf[0] : 0.0f, by = L.ubarf ? L.ubarf[1] : 0.0f, bz = L.ubarf ? L.ubarf[2] : 0.0f;
    collide2(g, L.kf, L.fsf, L.finv_rho0, bx, by, bz);
}

struct CellGeom {
    int x, y, z;
    int dxm, dxp, dym, dyp, dzm, dzp;  // neighbour offsets with periodic wrap
};

__device__ __forceinline__ int nb_off(const CellGeom &c, int q) {
    int o = 0;
    if (cx(q) < 0) o += c.dxm;
    if (cx(q) > 0) o += c.dxp;
    if (cy(q) < 0) o += c.dym;
    if (cy(q) > 0) o += c.dyp;
    if (cz(q) < 0) o += c.dzm;
    if (cz(q) > 0) o += c.dzp;
    return o;
}

// Coordinates of cell idx and its neighbour offsets, wrapped on every face
// (on a non-periodic face the cell is a wall and the wrapped neighbour is
// never used, but every index stays inside the lattice).
__device__ __forceinline__ CellGeom cell_geom(const LatDev &L, int idx) {
    CellGeom cg;
    const uint32_t yz = L.divx.div((uint32_t)idx);
    cg.x = idx - (int)yz * L.nx;
    cg.z = (int)L.divxy.div((uint32_t)idx);
    cg.y = (int)yz - cg.z * L.ny;
    const int sy = L.nx, sz = L.nx * L.ny;
    cg.dxm = cg.x == 0 ? L.nx - 1 : -1;
    cg.dxp = cg.x == L.nx - 1 ? -(L.nx - 1) : 1;
    cg.dym = cg.y == 0 ? (L.ny - 1) * sy : -sy;
    cg.dyp = cg.y == L.ny - 1 ? -(L.ny - 1) * sy : sy;
    cg.dzm = cg.z == 0 ? (L.nz - 1) * sz : -sz;
    cg.dzp = cg.z == L.nz - 1 ? -(L.nz - 1) * sz : sz;
    return cg;
}

template <bool SINGLE>
__device__ __forceinline__ int tile_lattice(const SweepArgs &a, int tile) {
    if (SINGLE) return 0;
    if (a.tile_lat) return a.tile_lat[tile];
    int lo = 0, hi = a.nlat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// L2 prefetch of the populations a later tile of the direct sweep reads
// (cp.async.bulk.prefetch: one asynchronous bulk request per plane, no
// registers held, no completion to wait for).  Thread q < 19 of the block
// covers plane q: on even steps the tile's own range, on odd steps the range
// shifted by the offset of x + c_q (the plane q pulls come from), widened by
// a few cells for the row-end wraps and rounded out to 16 bytes.  The ranges
// lie in the population arena: every plane is followed by the next one, and
// the arena's guard bands exceed the largest shift.
template <int PREC, int ODD, bool SINGLE>
__device__ __forceinline__ void prefetch_tile(const SweepArgs &a, int tile, int tcells) {
    const int q = (int)threadIdx.x;
    if (q >= Q || tile >= a.ntiles) return;
    const int li = tile_lattice<SINGLE>(a, tile);
    const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
    const long long start = (long long)(tile - L.tile0) * tcells;
    const long long cnt = min((long long)tcells, (long long)L.n - start);
    if (cnt <= 0) return;
    constexpr int EB = (int)sizeof(typename Store<PREC>::T);
    const long long e0 = L.f_off + (long long)q * L.npad + start + (ODD ? L.off[q] : 0) - 8;
    const uintptr_t b0 = (reinterpret_cast<uintptr_t>(a.f) + (uintptr_t)(e0 * EB)) & ~(uintptr_t)15;
    const uintptr_t b1 = (reinterpret_cast<uintptr_t>(a.f) + (uintptr_t)((e0 + cnt + 16) * EB) + 15) & ~(uintptr_t)15;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
}

// Per-thread partial sums of force and torque.  FP64 lattices keep them in
// FP64.  The FP32/FP16/BF16 lattices keep them as double-floats: GB300 issues
// FP64 arithmetic at a small fraction of its FP32 rate, and a single lane's
// FP64 chain on the sweep's critical path stalls the whole sweep, so the
// partials are compensated FP32 sums (about 48 significant bits) and only the
// global accumulators are FP64.
// float -> double by bit manipulation (exact for every float): GB300 issues
// the conversion instruction on its FP64 pipe, integer operations are free.
__device__ __forceinline__ double f2d_exact(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    uint64_t bits;
    if (e == 0xFFu) {
        bits = sign | (0x7FFull << 52) | ((uint64_t)m << 29);
    } else if (e != 0) {
        bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
    } else if (m == 0) {
        bits = sign;
    } else {  // subnormal: m 2^-149 with the leading one of m at bit p
        const int p = 31 - __clz((int)m);
        bits = sign | ((uint64_t)(p + 874) << 52) | ((uint64_t)((m << (23 - p)) & 0x7FFFFFu) << 29);
    }
    return __longlong_as_double((long long)bits);
}

template <int PREC> struct Acc {
    using V = df;
    // add to an FP64 accumulator: the two parts as two exact FP64 atomics
    // (the additions happen in the L2, not on the SM's FP64 pipe)
    static __device__ __forceinline__ void atomic_add(double *g, V x) {
        atomicAdd(g, f2d_exact(x.hi));
        if (x.lo != 0.f) atomicAdd(g, f2d_exact(x.lo));
    }
    static __device__ __forceinline__ V zero() { return {0.f, 0.f}; }
    static __device__ __forceinline__ V add(V x, V y) { return df_add(x, y); }
    static __device__ __forceinline__ V sub(V x, V y) { return df_add(x, df_neg(y)); }
    static __device__ __forceinline__ V mul(V x, V y) { return df_mul(x, y); }
    static __device__ __forceinline__ V from(double x) { return df_from_double(x); }
    static __device__ __forceinline__ V shfl_xor(V x, int o) {
        return {__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
    }
};
template <> struct Acc<LBM_F64> {
    using V = double;
    static __device__ __forceinline__ void atomic_add(double *g, V x) { atomicAdd(g, x); }
    static __device__ __forceinline__ V zero() { return 0.0; }
    static __device__ __forceinline__ V add(V x, V y) { return x + y; }
    static __device__ __forceinline__ V sub(V x, V y) { return x - y; }
    static __device__ __forceinline__ V mul(V x, V y) { return x * y; }
    static __device__ __forceinline__ V from(double x) { return x; }
    static __device__ __forceinline__ V shfl_xor(V x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
};

// Add nv components to this thread's partial sum for `key` (a body or a
// wall).  A thread holds one key at a time; meeting another key first hands
// the held partial to the global accumulators.
template <int PREC>
__device__ __forceinline__ void tacc_add(const SweepArgs &a, uint32_t *tkey, typename Acc<PREC>::V *tval,
                                         uint32_t key, const typename Acc<PREC>::V *v, int nv) {
    using A = Acc<PREC>;
    if (*tkey != key) {
        if (*tkey != SLOT_EMPTY) {
            double *g = global_acc(a, *tkey);
            const int nk = (*tkey & KEY_WALL) ? 3 : 6;
            for (int k = 0; k < nk; ++k) A::atomic_add(g + k, tval[k]);
        }
        *tkey = key;
        for (int k = 0; k < 6; ++k) tval[k] = A::zero();
    }
    for (int k = 0; k < nv; ++k) tval[k] = A::add(tval[k], v[k]);
}

// Momentum handed over by the links of one cell to one body or wall
// (Eq. TransferredMomentum): the link momentum (2 f~_q - 6 w_q rho0 c_q.u_s) c_q
// is split into the small part (2 g~_q - 6 w_q rho0 c_q.u_s) c_q, g~ the stored
// post-collision offset (of the order of the deviation from rest), summed in
// the compute precision over the cell's at most 18 links, and the constant
// part 2 w_q rho0 c_q = (rho0/18) (36 w_q) c_q, whose sum over the links in
// `mask` is rho0/18 times an exact integer vector.  F = small + constant.
template <int PREC, class C>
__device__ __forceinline__ void link_force(const LatDev &L, const C (&small)[3], uint32_t mask,
                                           typename Acc<PREC>::V F[3]) {
    int n[3] = {0, 0, 0};
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if ((mask >> q) & 1u) {
            const int w36 = q <= 6 ? 2 : 1;
            n[0] += cx(q) * w36;
            n[1] += cy(q) * w36;
            n[2] += cz(q) * w36;
        }
    if constexpr (PREC == LBM_F64) {
        for (int k = 0; k < 3; ++k) F[k] = small[k] + L.rho18 * (double)n[k];
    } else {
        const df r18 = {L.rho18f[0], L.rho18f[1]};
        for (int k = 0; k < 3; ++k) F[k] = df_add_f(df_mul_f(r18, (float)n[k]), small[k]);
    }
}

// Lever arm r_F = x_F - x_C of fluid cell (x, y, z) from body p's centre,
// minimum image on periodic axes: FP64 on FP64 lattices, else a double-float
// from the body's FP32 record.
template <int PREC>
__device__ __forceinline__ void lever_arm(const SweepArgs &a, const LatDev &L, uint32_t p, int x, int y, int z,
                                          typename Acc<PREC>::V r[3]) {
    const int xs[3] = {x, y, z}, ns[3] = {L.nx, L.ny, L.nz}, per[3] = {L.px, L.py, L.pz};
    if constexpr (PREC == LBM_F64) {
        for (int k = 0; k < 3; ++k) r[k] = min_image((double)xs[k] - a.P.pos[3 * (size_t)p + k], ns[k], per[k]);
    } else {
        const float *bf = a.P.bodyf + BF_STRIDE * (size_t)p;
        for (int k = 0; k < 3; ++k) {
            df d = two_sum((float)xs[k], -bf[BF_POS + k]);
            d = df_add_f(d, -bf[BF_POSLO + k]);
            if (per[k]) {
                if (d.hi > 0.5f * (float)ns[k])
                    d = df_add_f(d, -(float)ns[k]);
                else if (d.hi < -0.5f * (float)ns[k])
                    d = df_add_f(d, (float)ns[k]);
            }
            r[k] = d;
        }
    }
}

// Hand a body's per-cell momentum F and torque r_F x F to the partial sums
// (the torque of link q is (r_F + c_q) x dF_q = r_F x dF_q since dF_q || c_q).
template <int PREC>
__device__ __forceinline__ void body_add(const SweepArgs &a, uint32_t *tkey, typename Acc<PREC>::V *tval,
                                         uint32_t key, const typename Acc<PREC>::V F[3],
                                         const typename Acc<PREC>::V r[3]) {
    using A = Acc<PREC>;
    typename A::V v[6] = {F[0], F[1], F[2],
                          A::sub(A::mul(r[1], F[2]), A::mul(r[2], F[1])),
                          A::sub(A::mul(r[2], F[0]), A::mul(r[0], F[2])),
                          A::sub(A::mul(r[0], F[1]), A::mul(r[1], F[0]))};
    tacc_add<PREC>(a, tkey, tval, key, v, 6);
}

// Velocity bounce-back of one link (Eq. LBMMovWall) and its momentum
// exchange (Eqs. TransferredMomentum, LBMhydrodynForce), generic over the
// neighbour (either wall layer or any body), in FP64.  ft is the
// post-collision offset f~_q - w_q rho0 of the fluid cell; returns the offset
// of the reflected population f~_q - 6 w_q rho0 c_q.u_s.  The momentum
// (2 f~_q - 6 w_q rho0 c_q.u_s) c_q, and its torque (x_s - x_C) x dF about the
// body centre, go into this thread's partial-sum entry.  Used for links to a
// second body of the same cell (the first body's links are handled inline).
template <int PREC>
__device__ __noinline__ double bounce_link(const SweepArgs &a, const LatDev &L, int li, int q, int nb,
                                           int xs, int ys, int zs, double ft, uint32_t *tkey,
                                           typename Acc<PREC>::V *tval) {
    using A = Acc<PREC>;
    const uint32_t id = a.pid[L.c_off + nb];
    double us[3] = {0.0, 0.0, 0.0}, r[3] = {0.0, 0.0, 0.0};
    uint32_t key = SLOT_EMPTY;
    if (id == PID_WALL_YLO) {
        us[0] = L.wlo[0]; us[1] = L.wlo[1]; us[2] = L.wlo[2];
        key = KEY_WALL | ((uint32_t)li << 1);
    } else if (id == PID_WALL_YHI) {
        us[0] = L.whi[0]; us[1] = L.whi[1]; us[2] = L.whi[2];
        key = KEY_WALL | ((uint32_t)li << 1) | 1u;
    } else if (id < PID_WALL) {
        const double *pos = a.P.pos + 3 * (size_t)id;
        const double *U = a.P.vel + 3 * (size_t)id;
        const double *W = a.P.om + 3 * (size_t)id;
        r[0] = min_image((double)xs - pos[0], L.nx, L.px);
        r[1] = min_image((double)ys - pos[1], L.ny, L.py);
        r[2] = min_image((double)zs - pos[2], L.nz, L.pz);
        us[0] = U[0] + (W[1] * r[2] - W[2] * r[1]);
        us[1] = U[1] + (W[2] * r[0] - W[0] * r[2]);
        us[2] = U[2] + (W[0] * r[1] - W[1] * r[0]);
        key = id;
    }
    const int qx = c_cx[q], qy = c_cy[q], qz = c_cz[q];
    const double w = c_w[q];
    const double cu = qx * us[0] + qy * us[1] + qz * us[2];
    const double dbb = 6.0 * w * L.rho0 * cu;
    if (key != SLOT_EMPTY) {
        const double mag = 2.0 * (ft + w * L.rho0) - dbb;
        double v[6];
        v[0] = mag * qx;
        v[1] = mag * qy;
        v[2] = mag * qz;
        v[3] = r[1] * v[2] - r[2] * v[1];
        v[4] = r[2] * v[0] - r[0] * v[2];
        v[5] = r[0] * v[1] - r[1] * v[0];
        typename A::V va[6];
        for (int k = 0; k < 6; ++k) va[k] = A::from(v[k]);
        tacc_add<PREC>(a, tkey, tval, key, va, 6);
    }
    return ft - dbb;
}

// Links of a near-obstacle cell to bodies other than the first one met and to
// a second moving wall layer (rare): the sweep has stored the unbounced
// post-collision value in the bounce-back slot opp(q) of x; bounce_link turns
// it into the reflected value and books the momentum.  Kept out of the link
// loop, so that the loop makes no calls.
template <int PREC>
__device__ __noinline__ void other_links(const SweepArgs &a, const LatDev &L, int li, int idx, uint32_t mask,
                                         uint32_t *tkey, typename Acc<PREC>::V *tval, Rnd<PREC> *rnd) {
    using S = Store<PREC>;
    using T = typename S::T;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    const CellGeom cg = cell_geom(L, idx);
    for (uint32_t m = mask; m; m &= m - 1) {
        const int q = __ffs(m) - 1;
        const int qx = c_cx[q], qy = c_cy[q], qz = c_cz[q];
        const int qo = q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1);
        int nb = 0;
        nb += qx < 0 ? cg.dxm : (qx > 0 ? cg.dxp : 0);
        nb += qy < 0 ? cg.dym : (qy > 0 ? cg.dyp : 0);
        nb += qz < 0 ? cg.dzm : (qz > 0 ? cg.dzp : 0);
        T *slot = base + qo * np + idx;
        const double v = bounce_link<PREC>(a, L, li, q, idx + nb, wrapc(cg.x + qx, L.nx), wrapc(cg.y + qy, L.ny),
                                           wrapc(cg.z + qz, L.nz), (double)S::ldg(slot), tkey, tval);
        S::stg(slot, (typename S::C)v, rnd->next());
    }
}

// Fluid cell next to walls or obstacles: neighbour flags decide where each
// population is read from (odd steps) and which outgoing populations are
// bounced back.
// Shared-memory staging of a tile (see sweep_staged): W elements per window,
// A elements per 16 bytes (the bulk-copy alignment unit).
template <int PREC> struct StageCfg {
    using T = typename Store<PREC>::T;
    static constexpr int TILE = 256;
    static constexpr int A = 16 / (int)sizeof(T);
    static constexpr int W = TILE + A;
    static constexpr int S = sizeof(T) == 8 ? 2 : 3;  // pipeline depth (tiles)
    // 19 population windows, then the tile's TILE flag bytes
    static constexpr int STAGE_ELEMS = Q * W + TILE / (int)sizeof(T);
    static constexpr int SMEM = S * STAGE_ELEMS * (int)sizeof(T);
};

// Per-thread prefetch ring (see sweep_ring): one column of ROWS words per
// thread and ring slot; a word holds one population (a 16-bit population
// sits in the half given by the parity of its element index).
template <int PREC> struct RingCfg {
    using T = typename Store<PREC>::T;
    using Word = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    static constexpr int TILE = 256;
    static constexpr int D = 2;             // tiles prefetched ahead of the one being updated
    static constexpr int ROWS = Q + 1;      // 19 populations and the word holding the flag byte
    static constexpr int SLOT = ROWS * TILE;
    static constexpr int SMEM = (D + 1) * SLOT * (int)sizeof(Word);
};

template <int PREC>
__device__ __forceinline__ typename Store<PREC>::C ring_value(const typename RingCfg<PREC>::Word *col, int q,
                                                              int parity) {
    using S = Store<PREC>;
    using T = typename S::T;
    const auto w = col[q * RingCfg<PREC>::TILE];
    if constexpr (sizeof(T) == 2) {
        const unsigned short h = (unsigned short)(parity ? (w >> 16) : (w & 0xFFFFu));
        T v;
        memcpy(&v, &h, 2);
        return S::ld(&v);
    } else {
        T v;
        memcpy(&v, &w, sizeof(T));
        return S::ld(&v);
    }
}

// Population source of the near-obstacle path: VIEW 0 reads global memory,
// 1 the bulk-copy stage window `src`, 2 the thread's ring column `src`, 3
// finds the bulk pull values in g already (the direct sweep loads them with
// the flag byte); the populations bounced off obstacles in the previous step
// always come from global memory.  Inlined: the caller's arrays stay in
// registers.
template <int PREC, int ODD, int VIEW>
__device__ __forceinline__ void near_cell(const SweepArgs &a, const LatDev &L, int li, int idx,
                                          uint32_t *tkey, typename Acc<PREC>::V *tval, const void *src,
                                          typename Store<PREC>::C (&g)[Q], uint32_t seed) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Cfg = StageCfg<PREC>;
    const CellGeom cg = cell_geom(L, idx);
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    const T *stage = reinterpret_cast<const T *>(src);
    const typename RingCfg<PREC>::Word *col = reinterpret_cast<const typename RingCfg<PREC>::Word *>(src);
    // the flags pass keeps, per fluid cell, which neighbours are wall or
    // obstacle cells, which of them are wall-layer cells and which belong to
    // the first body met in q order (p0)
    const uint64_t lk = a.links[L.c_off + idx];
    const uint32_t solid = (uint32_t)lk & LK_MASK;            // bit q: x + c_q is a wall or obstacle cell
    const uint32_t wall = (uint32_t)(lk >> LK_WALL) & LK_MASK;  // bit q: x + c_q is a wall-layer cell
    const uint32_t m0 = (uint32_t)(lk >> LK_BODY) & LK_MASK;    // bit q: x + c_q is a cell of body p0
    // free-slip wall links carry the wall bit without the solid bit
    const uint32_t fsl = wall & ~solid, wbb = wall & solid;
    // Obstacle links: the first body met (p0) has its motion loaded once and
    // its links are bounced inline in the compute precision, their momentum
    // summed per cell; links to any further body take bounce_link.
    const uint32_t p0 = m0 ? a.nbody[L.c_off + idx] : SLOT_EMPTY;
    // body p0: lever arm r_F of this cell (compute precision), velocity U and
    // angular velocity W
    using A = Acc<PREC>;
    C rc[3] = {0, 0, 0}, bU[3] = {0, 0, 0}, bW[3] = {0, 0, 0};
    if (p0 != SLOT_EMPTY) {
        typename A::V rF[3];
        lever_arm<PREC>(a, L, p0, cg.x, cg.y, cg.z, rF);
        for (int k = 0; k < 3; ++k) {
            if constexpr (PREC == LBM_F64) {
                rc[k] = rF[k];
                bU[k] = a.P.vel[3 * (size_t)p0 + k];
                bW[k] = a.P.om[3 * (size_t)p0 + k];
            } else {
                rc[k] = rF[k].hi;
                bU[k] = a.P.bodyf[BF_STRIDE * (size_t)p0 + BF_U + k];
                bW[k] = a.P.bodyf[BF_STRIDE * (size_t)p0 + BF_W + k];
            }
        }
    }
    if (VIEW == 3) {
        if (ODD) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if ((solid >> opp(q)) & 1u) g[q] = S::ldg(base + q * np + idx);
        }
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int p = opp(q);
            if (!ODD) {
                if (VIEW == 1) g[q] = S::ld(stage + q * Cfg::W + threadIdx.x);
                else if (VIEW == 2) g[q] = ring_value<PREC>(col, q, idx & 1);
                else g[q] = S::ldg(base + q * np + idx);
            } else if ((solid >> p) & 1u) {
                g[q] = S::ldg(base + q * np + idx);
            } else if (VIEW == 1) {
                g[q] = S::ld(stage + q * Cfg::W + (L.off[p] & (Cfg::A - 1)) + threadIdx.x);
            } else if (VIEW == 2) {
                g[q] = ring_value<PREC>(col, q, (idx + nb_off(cg, p)) & 1);
            } else {
                g[q] = S::ldg(base + p * np + idx + nb_off(cg, p));
            }
        }
    }
    collide_lat<C>(g, L);
    // Wall links are bounced inline as well.  The y = 0 and y = ny-1 layers of
    // a non-periodic y axis move; their links (wmain: the layer met first)
    // hand momentum to that wall; any other wall layer rests.  A cell touching
    // both moving layers (ny = 3) sends the second layer's links through
    // bounce_link.
    uint32_t wlo = 0, whi = 0;
    if (wbb && !L.py) {
#pragma unroll
        for (int q = 1; q < Q; ++q)
            if ((wbb >> q) & 1u) {
                if (cg.y + cy(q) == 0) wlo |= 1u << q;
                else if (cg.y + cy(q) == L.ny - 1) whi |= 1u << q;
            }
    }
    const int wside = wlo ? 0 : (whi ? 1 : -1);
    const uint32_t wmain = wlo ? wlo : whi;
    const uint32_t wrest = wbb & ~(wlo | whi);
    const LatPar<C> lp(L);
    const C rho0c = lp.rho0;
    const C *uw = wside == 1 ? lp.whi : lp.wlo;
    C sw[3] = {0, 0, 0}, sb[3] = {0, 0, 0};  // small parts of the wall / body p0 momentum
    Rnd<PREC> rnd(seed, L.c_off + idx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if ((wmain >> q) & 1u) {
            C cu = 0;
            if (cx(q)) cu += cx(q) > 0 ? uw[0] : -uw[0];
            if (cy(q)) cu += cy(q) > 0 ? uw[1] : -uw[1];
            if (cz(q)) cu += cz(q) > 0 ? uw[2] : -uw[2];
            const C dbb = C(6.0 * wq(q)) * rho0c * cu;
            const C sm = C(2) * g[q] - dbb;
            if (cx(q)) sw[0] += cx(q) > 0 ? sm : -sm;
            if (cy(q)) sw[1] += cy(q) > 0 ? sm : -sm;
            if (cz(q)) sw[2] += cz(q) > 0 ? sm : -sm;
            S::stg(base + opp(q) * np + idx, g[q] - dbb, rnd.next());
        } else if ((wrest >> q) & 1u) {
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        } else if ((m0 >> q) & 1u) {
            // velocity bounce-back off body p0 (Eq. LBMMovWall): u_s at the
            // obstacle cell x_F + c_q, lever arm r_F + c_q
            const C r0 = rc[0] + C(cx(q)), r1 = rc[1] + C(cy(q)), r2 = rc[2] + C(cz(q));
            const C us0 = bU[0] + (bW[1] * r2 - bW[2] * r1);
            const C us1 = bU[1] + (bW[2] * r0 - bW[0] * r2);
            const C us2 = bU[2] + (bW[0] * r1 - bW[1] * r0);
            C cu = 0;
            if (cx(q)) cu += cx(q) > 0 ? us0 : -us0;
            if (cy(q)) cu += cy(q) > 0 ? us1 : -us1;
            if (cz(q)) cu += cz(q) > 0 ? us2 : -us2;
            const C dbb = C(6.0 * wq(q)) * rho0c * cu;
            const C sm = C(2) * g[q] - dbb;
            if (cx(q)) sb[0] += cx(q) > 0 ? sm : -sm;
            if (cy(q)) sb[1] += cy(q) > 0 ? sm : -sm;
            if (cz(q)) sb[2] += cz(q) > 0 ? sm : -sm;
            S::stg(base + opp(q) * np + idx, g[q] - dbb, rnd.next());
        } else if ((solid >> q) & 1u) {
            // another body (or the second moving wall layer): the unbounced
            // value goes to the bounce-back slot now, other_links rewrites it
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        } else if ((fsl >> q) & 1u) {
            // free-slip wall (Eq. FreeSlipBC): the components whose wall layer
            // the link crosses are reversed; the value arrives at x + c_q minus
            // those components, in the reflected direction r
            const bool ax = cx(q) != 0 && !L.px && (cg.x + cx(q) == 0 || cg.x + cx(q) == L.nx - 1);
            const bool ay = cy(q) != 0 && !L.py && (cg.y + cy(q) == 0 || cg.y + cy(q) == L.ny - 1);
            const bool az = cz(q) != 0 && !L.pz && (cg.z + cz(q) == 0 || cg.z + cz(q) == L.nz - 1);
            const int r = c_qidx[(ax ? -cx(q) : cx(q)) + 1 + 3 * ((ay ? -cy(q) : cy(q)) + 1) +
                                 9 * ((az ? -cz(q) : cz(q)) + 1)];
            if (!ODD) {
                // the arrival cell pulls it next step through the wall cell
                // x + (crossed components of c_q), whose slots are otherwise unused
                const int wcell = idx + (ax ? cx(q) : 0) + (ay ? cy(q) * L.nx : 0) + (az ? cz(q) * L.nx * L.ny : 0);
                S::stg(base + (long long)opp(r) * np + wcell, g[q], rnd.next());
            } else {
                int off = 0;
                if (cx(q) && !ax) off += cx(q) > 0 ? cg.dxp : cg.dxm;
                if (cy(q) && !ay) off += cy(q) > 0 ? cg.dyp : cg.dym;
                if (cz(q) && !az) off += cz(q) > 0 ? cg.dzp : cg.dzm;
                S::stg(base + (long long)r * np + idx + off, g[q], rnd.next());
            }
        } else if (!ODD) {
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        } else {
            S::stg(base + q * np + idx + nb_off(cg, q), g[q], rnd.next());
        }
    }
    const uint32_t mo = solid & ~(m0 | wmain | wrest);
    if (mo) other_links<PREC>(a, L, li, idx, mo, tkey, tval, &rnd);
    if (m0) {
        typename A::V F[3], rF[3];
        link_force<PREC>(L, sb, m0, F);
        lever_arm<PREC>(a, L, p0, cg.x, cg.y, cg.z, rF);
        body_add<PREC>(a, tkey, tval, p0, F, rF);
    }
    if (wmain) {
        typename A::V F[3];
        link_force<PREC>(L, sw, wmain, F);
        tacc_add<PREC>(a, tkey, tval, KEY_WALL | ((uint32_t)li << 1) | (uint32_t)wside, F, 3);
    }
}

// Fluid cell whose only wall/obstacle neighbours are the moving wall layer
// y = 0 (SIDE 0) or y = ny-1 (SIDE 1): the bounced directions are the five with
// c_y = -1 (resp. +1), known at compile time.  On odd steps the five
// populations arriving from the layer are the ones the previous step bounced
// into slot q of x itself.  Out of line, with its own loads, so that the
// caller's bulk path keeps its registers.
template <int PREC, int ODD, int SIDE>
__device__ __noinline__ void wall_cell(const SweepArgs &a, const LatDev &L, int li, int idx,
                                       uint32_t *tkey, typename Acc<PREC>::V *tval, uint32_t seed) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    C g[Q];
    CellGeom cg;
    if (ODD) {
        cg = cell_geom(L, idx);
#pragma unroll
        for (int q = 0; q < Q; ++q)
            g[q] = (q != 0 && (SIDE == 0 ? cy(q) > 0 : cy(q) < 0)) ? S::ldg(base + q * np + idx)
                                                                  : S::ldg(base + opp(q) * np + idx + nb_off(cg, opp(q)));
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) g[q] = S::ldg(base + q * np + idx);
    }
    collide_lat<C>(g, L);
    const LatPar<C> lp(L);
    const C *uw = SIDE == 0 ? lp.wlo : lp.whi;
    const C u0 = uw[0], u1 = uw[1], u2 = uw[2], rho0c = lp.rho0;
    C sw[3] = {0, 0, 0};
    uint32_t mask = 0;
    Rnd<PREC> rnd(seed, L.c_off + idx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (SIDE == 0 ? cy(q) < 0 : cy(q) > 0) {
            C cu = 0;
            if (cx(q)) cu += cx(q) > 0 ? u0 : -u0;
            cu += cy(q) > 0 ? u1 : -u1;
            if (cz(q)) cu += cz(q) > 0 ? u2 : -u2;
            const C dbb = C(6.0 * wq(q)) * rho0c * cu;
            S::stg(base + opp(q) * np + idx, g[q] - dbb, rnd.next());
            const C sm = C(2) * g[q] - dbb;
            if (cx(q)) sw[0] += cx(q) > 0 ? sm : -sm;
            sw[1] += cy(q) > 0 ? sm : -sm;
            if (cz(q)) sw[2] += cz(q) > 0 ? sm : -sm;
            mask |= 1u << q;
        } else if (!ODD) {
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        } else {
            S::stg(base + q * np + idx + nb_off(cg, q), g[q], rnd.next());
        }
    }
    typename Acc<PREC>::V F[3];
    link_force<PREC>(L, sw, mask, F);
    tacc_add<PREC>(a, tkey, tval, KEY_WALL | ((uint32_t)li << 1) | (uint32_t)SIDE, F, 3);
}

// Fluid cell with fluid neighbours only.
template <int PREC, int ODD>
__device__ __forceinline__ void bulk_cell(const SweepArgs &a, const LatDev &L, int idx, uint32_t seed) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    CellGeom cg;
    if (ODD) cg = cell_geom(L, idx);
    C g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            g[q] = S::ldg(base + q * np + idx);
        else
            g[q] = S::ldg(base + opp(q) * np + idx + nb_off(cg, opp(q)));
    }
    collide_lat<C>(g, L);
    Rnd<PREC> rnd(seed, L.c_off + idx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        else
            S::stg(base + q * np + idx + nb_off(cg, q), g[q], rnd.next());
    }
}

// Minimum resident blocks of 256 threads per SM: 3 leaves 80 registers per
// thread, enough for the bulk path to keep all 19 populations and their
// addresses in registers without spilling.
template <int PREC> struct SweepBounds { static constexpr int MINB = 3; };
template <> struct SweepBounds<LBM_F64> { static constexpr int MINB = 2; };

// Hand the per-thread partial sums to the global accumulators, warp by warp
// and key by key (body or wall): the lanes holding the key add their partials
// in a butterfly over the warp (the others add zero), and the lowest of them
// issues one FP64 atomic per component.  No block barrier, so blocks without
// wall or obstacle links never wait on each other's warps; warps without any
// key leave after one vote.
template <int PREC>
__device__ __forceinline__ void flush_forces(const SweepArgs &a, uint32_t *tkey,
                                             typename Acc<PREC>::V (*tval)[6]) {
    using A = Acc<PREC>;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    uint32_t key = tkey[threadIdx.x];
    for (uint32_t pending = __ballot_sync(0xffffffffu, key != SLOT_EMPTY); pending;
         pending = __ballot_sync(0xffffffffu, key != SLOT_EMPTY)) {
        const int leader = __ffs(pending) - 1;
        const uint32_t k0 = __shfl_sync(0xffffffffu, key, leader);
        const bool mine = key == k0;
        const int nv = (k0 & KEY_WALL) ? 3 : 6;
        double *g = global_acc(a, k0);
        for (int k = 0; k < nv; ++k) {
            typename A::V v = mine ? tval[threadIdx.x][k] : A::zero();
#pragma unroll
            for (int o = 16; o; o >>= 1) v = A::add(v, A::shfl_xor(v, o));
            if (lane == leader) A::atomic_add(g + k, v);
        }
        if (mine) key = SLOT_EMPTY;
    }
}

// Direct sweep, one cell per thread: plain stream-collide for bulk cells,
// the wall and near-obstacle paths for cells flagged F_YLO/F_YHI or F_NEAR.
// SINGLE: one lattice, whose parameters travel in the kernel's parameter
// space (a.lat0) and are read as constant-bank operands; otherwise each tile
// finds its lattice in the global table by binary search on tile0.
template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_kernel(const __grid_constant__ SweepArgs a) {
    pdl_enter();
    const uint32_t seed = PREC == LBM_BF16_OFFSET ? step_seed(a.tick) : 0u;
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    __shared__ uint32_t tkey[256];
    __shared__ typename Acc<PREC>::V tval[256][6];
    tkey[threadIdx.x] = SLOT_EMPTY;

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        if (a.pf_ahead[ODD]) prefetch_tile<PREC, ODD, SINGLE>(a, tile + a.pf_ahead[ODD], (int)blockDim.x);
        const int li = tile_lattice<SINGLE>(a, tile);
        const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
        const int idx = (tile - L.tile0) * blockDim.x + threadIdx.x;
        if (idx >= L.n) continue;
        if (a.tbits && !((a.tbits[tile >> 5] >> (tile & 31)) & 1u)) {
            // a tile of bulk fluid cells only (uniform per block): no flag read
            bulk_cell<PREC, ODD>(a, L, idx, seed);
            continue;
        }
        T *base = reinterpret_cast<T *>(a.f) + L.f_off;
        const long long np = L.npad;
        // the 19 populations are read at the bulk pull addresses, which are in
        // range for every cell, in the same round trip as the flag byte
        C g[Q];
        CellGeom cg;
        if (ODD) {
            cg = cell_geom(L, idx);
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = S::ldg(base + opp(q) * np + idx + nb_off(cg, opp(q)));
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = S::ldg(base + q * np + idx);
        }
        const uint8_t fl = a.flags[L.c_off + idx];
        if (fl & F_SOLID) continue;
        if (fl & (F_YLO | F_YHI)) {
            if (fl & F_YLO)
                wall_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x], seed);
            else
                wall_cell<PREC, ODD, 1>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x], seed);
            continue;
        }
        if (fl & F_NEAR) {
            if (a.near_list) continue;  // split sweep: the near kernel updates it
            near_cell<PREC, ODD, 3>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x], nullptr, g, seed);
            continue;
        }
        collide_lat<C>(g, L);
        Rnd<PREC> rnd(seed, L.c_off + idx);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!ODD)
                S::stg(base + opp(q) * np + idx, g[q], rnd.next());
            else
                S::stg(base + q * np + idx + nb_off(cg, q), g[q], rnd.next());
        }
    }
    flush_forces<PREC>(a, tkey, tval);
}

// ---------------------------------------------------------------------------
// Direct sweep over groups of V consecutive cells per thread (V = 2 or 4).
// A thread issues the loads of all its cells before it collides any of them,
// so V times the bytes of the one-cell sweep are in flight per thread, and it
// moves the V values of one population plane with one vector access (4, 8 or
// 16 bytes) wherever they are contiguous and aligned: every plane on even
// steps (a cell's own slots), and on odd steps the planes of directions
// without an x component, whose neighbour offsets are whole rows -- a group
// x0 .. x0+V-1 with x0 a multiple of V stays an aligned group when V divides
// nx.  Directions with an x component are moved element by element on odd
// steps, each cell with its own periodic wrap at the row ends.  A lattice
// whose nx is not a multiple of V, and the ragged last group of a lattice,
// take element accesses throughout.  The AA property holds as in the one-cell
// sweep: a thread reads and writes only its own cells' slots.  Groups whose
// cells are all bulk fluid run the collision on the packed values; a group
// with a wall, obstacle or near-obstacle cell takes the one-cell paths.
// ---------------------------------------------------------------------------

// V consecutive storage elements of one population plane, packed into 32-bit
// words (element k at bits 16(k&1) of word k/2 for the 16-bit forms, word k
// for FP32, words 2k, 2k+1 for FP64).  Element indices are compile-time after
// unrolling, so the packing folds into register moves and byte permutes.
template <int PREC, int V> struct Pack {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    static constexpr int EB = (int)sizeof(T);
    static constexpr int NW = V * EB / 4;
    static_assert(NW == 1 || NW == 2 || NW == 4, "a group of 4, 8 or 16 bytes");
    uint32_t w[NW];

    __device__ __forceinline__ void vload(const T *p) {
        if constexpr (NW == 1) {
            w[0] = __ldcs(reinterpret_cast<const unsigned int *>(p));
        } else if constexpr (NW == 2) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
            w[0] = v.x;
            w[1] = v.y;
        } else {
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(p));
            w[0] = v.x;
            w[1] = v.y;
            w[2] = v.z;
            w[3] = v.w;
        }
    }
    __device__ __forceinline__ void vstore(T *p) const {
        if constexpr (NW == 1)
            __stcs(reinterpret_cast<unsigned int *>(p), w[0]);
        else if constexpr (NW == 2)
            __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w[0], w[1]));
        else
            __stcs(reinterpret_cast<uint4 *>(p), make_uint4(w[0], w[1], w[2], w[3]));
    }
    // raw 16 bits into element k (16-bit forms)
    __device__ __forceinline__ void put16(int k, uint32_t h) {
        w[k >> 1] = (k & 1) ? __byte_perm(w[k >> 1], h, 0x5410) : __byte_perm(w[k >> 1], h, 0x3254);
    }
    __device__ __forceinline__ void eload(const T *p, int k) {
        if constexpr (EB == 2) {
            put16(k, __ldcs(reinterpret_cast<const unsigned short *>(p)));
        } else if constexpr (EB == 4) {
            w[k] = __ldcs(reinterpret_cast<const unsigned int *>(p));
        } else {
            const uint2 v = __ldcs(reinterpret_cast<const uint2 *>(p));
            w[2 * k] = v.x;
            w[2 * k + 1] = v.y;
        }
    }
    __device__ __forceinline__ void estore(T *p, int k) const {
        if constexpr (EB == 2)
            __stcs(reinterpret_cast<unsigned short *>(p), (unsigned short)((k & 1) ? w[k >> 1] >> 16 : w[k >> 1]));
        else if constexpr (EB == 4)
            __stcs(reinterpret_cast<unsigned int *>(p), w[k]);
        else
            __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w[2 * k], w[2 * k + 1]));
    }
    // elements 1 and 2 (V = 4) to p, p[0] and p[1] (an aligned pair)
    __device__ __forceinline__ void pstore12(T *p) const {
        if constexpr (EB == 2)
            __stcs(reinterpret_cast<unsigned int *>(p), __byte_perm(w[0], w[1], 0x5432));
        else if constexpr (EB == 4)
            __stcs(reinterpret_cast<uint2 *>(p), make_uint2(w[1], w[2]));
    }
    // the group shifted by one element: elements 1..V-1 of own then element 0
    // of nbr (up: nbr is the group at x + V), or element V-1 of nbr then
    // elements 0..V-2 of own (nbr is the group at x - V)
    __device__ __forceinline__ void shifted(bool up, const Pack &own, const Pack &nbr) {
        if constexpr (EB == 2) {
            if (up) {
                for (int j = 0; j < NW; ++j) w[j] = __byte_perm(own.w[j], j + 1 < NW ? own.w[j + 1] : nbr.w[0], 0x5432);
            } else {
                for (int j = 0; j < NW; ++j) w[j] = __byte_perm(j > 0 ? own.w[j - 1] : nbr.w[NW - 1], own.w[j], 0x5432);
            }
        } else {
            constexpr int E = EB / 4;  // words per element
            if (up) {
                for (int j = 0; j < NW; ++j) w[j] = j + E < NW ? own.w[j + E] : nbr.w[j + E - NW];
            } else {
                for (int j = 0; j < NW; ++j) w[j] = j >= E ? own.w[j - E] : nbr.w[NW - E + j];
            }
        }
    }
    __device__ __forceinline__ C get(int k) const {
        if constexpr (EB == 2)
            return S::from_bits((unsigned short)((k & 1) ? w[k >> 1] >> 16 : w[k >> 1]));
        else if constexpr (EB == 4)
            return __uint_as_float(w[k]);
        else
            return __hiloint2double((int)w[2 * k + 1], (int)w[2 * k]);
    }
    // elements k, k+1 (k even) as a pair in the compute precision (FP32 and
    // the 16-bit forms)
    __device__ __forceinline__ float2 get2(int k) const {
        if constexpr (PREC == LBM_F16_OFFSET) {
            return __half22float2(*reinterpret_cast<const __half2 *>(&w[k >> 1]));
        } else if constexpr (PREC == LBM_BF16_OFFSET) {
            const uint32_t x = w[k >> 1];
            return make_float2(__uint_as_float(x << 16), __uint_as_float(x & 0xffff0000u));
        } else {
            return make_float2(__uint_as_float(w[k]), __uint_as_float(w[k + 1]));
        }
    }
    // elements k, k+1 <- v (r0, r1: rounding bits of the BF16 form; `plain`:
    // no NaN among the two values, so the BF16 form rounds by integer adds)
    __device__ __forceinline__ void set2(int k, float2 v, uint32_t r0, uint32_t r1, bool plain) {
        if constexpr (PREC == LBM_F16_OFFSET) {
            const __half2 h = __float22half2_rn(v);
            w[k >> 1] = *reinterpret_cast<const uint32_t *>(&h);
        } else if constexpr (PREC == LBM_BF16_OFFSET) {
            if (plain) {
                // bf16_bits_sr of each value: add the rounding bits below the
                // kept 16 bits, keep the upper halves of both words
                w[k >> 1] = __byte_perm(__float_as_uint(v.x) + r0, __float_as_uint(v.y) + r1, 0x7632);
            } else {
                w[k >> 1] = (uint32_t)bf16_bits_sr(v.x, r0) | ((uint32_t)bf16_bits_sr(v.y, r1) << 16);
            }
        } else {
            w[k] = __float_as_uint(v.x);
            w[k + 1] = __float_as_uint(v.y);
        }
    }
    // element k <- v in the storage form (r16: rounding bits of the BF16 form)
    __device__ __forceinline__ void set(int k, C v, uint32_t r16) {
        if constexpr (EB == 2) {
            put16(k, S::bits(v, r16));
        } else if constexpr (EB == 4) {
            w[k] = __float_as_uint(v);
        } else {
            w[2 * k] = (uint32_t)__double2loint(v);
            w[2 * k + 1] = (uint32_t)__double2hiint(v);
        }
    }
};

// Offset of the neighbour x + c_q without its x part (rows and planes,
// periodic wrap included).
__device__ __forceinline__ int yz_off(const CellGeom &c, int q) {
    int o = 0;
    if (cy(q) < 0) o += c.dym;
    if (cy(q) > 0) o += c.dyp;
    if (cz(q) < 0) o += c.dzm;
    if (cz(q) > 0) o += c.dzp;
    return o;
}

// x part of that offset for cell k of an aligned group starting at c.x: the
// neighbour wraps only for the first cell of the row going -x and the last
// cell going +x.
template <int V>
__device__ __forceinline__ int x_off(const CellGeom &c, const LatDev &L, int q, int k) {
    if (cx(q) > 0) return (k == V - 1 && c.x + V == L.nx) ? 1 - L.nx : 1;
    if (cx(q) < 0) return k == 0 ? c.dxm : -1;
    return 0;
}

// A group with a wall, obstacle or near-obstacle cell: its bulk and wall
// cells one at a time through the one-cell paths (each loading its own
// populations), its near-obstacle cells left to the warp's near pass (bit k
// of the result: cell idx0 + k).
template <int PREC, int ODD, int V>
__device__ __forceinline__ uint32_t group_mixed(const SweepArgs &a, const LatDev &L, int li, int idx0, uint32_t fl,
                                             uint32_t seed, uint32_t *tkey, typename Acc<PREC>::V *tval) {
    uint32_t deferred = 0;
#pragma unroll 1
    for (int k = 0; k < V; ++k) {
        const int idx = idx0 + k;
        if (idx >= L.n) break;
        const uint8_t f = (uint8_t)(fl >> (8 * k));
        if (f & F_SOLID) continue;
        if (f & (F_YLO | F_YHI)) {
            if (f & F_YLO)
                wall_cell<PREC, ODD, 0>(a, L, li, idx, tkey, tval, seed);
            else
                wall_cell<PREC, ODD, 1>(a, L, li, idx, tkey, tval, seed);
        } else if (f & F_NEAR) {
            if (!a.near_list) deferred |= 1u << k;  // split sweep: the near kernel updates it
        } else {
            bulk_cell<PREC, ODD>(a, L, idx, seed);
        }
    }
    return deferred;
}

// The warp's near-obstacle cells, one per lane: the deferred cells of all
// lanes (bit k of `deferred`: cell idx0 + k of this lane's group) are listed
// in the warp's slice of shared memory in lane order and taken 32 at a time.
// A near cell's update touches only its own slots (AA), so doing it after the
// bulk cells of its warp changes nothing but the order of independent writes;
// run cell by cell inside the groups, the long near path would be issued up
// to V times per warp.  Called by the whole warp.
template <int PREC, int ODD, int V>
__device__ __forceinline__ void near_pass(const SweepArgs &a, const LatDev &L, int li, int idx0, uint32_t deferred,
                                       int *list, uint32_t seed, uint32_t *tkey, typename Acc<PREC>::V *tval) {
    using C = typename Store<PREC>::C;
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(deferred);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int w = incl - cnt;
    for (uint32_t m = deferred; m; m &= m - 1) list[w++] = idx0 + __ffs(m) - 1;
    __syncwarp();
#pragma unroll 1
    for (int j = lane; j < total; j += 32) {
        C g[Q];
        near_cell<PREC, ODD, 0>(a, L, li, list[j], tkey, tval, nullptr, g, seed);
    }
    __syncwarp();
}

// Loads of a group at the bulk pull addresses (odd steps: plane opp(q) at
// x - c_q); WALL = 0 / 1 reads the directions arriving from the moving wall
// layer y = 0 / y = ny-1 from the cell's own slot q instead (the previous
// step bounced them there), WALL = -1 none.
template <int PREC, int ODD, int V, int WALL>
__device__ __forceinline__ void group_load(const LatDev &L, typename Store<PREC>::T *base, long long np, int idx0,
                                           const CellGeom &cg, Pack<PREC, V> (&pk)[Q]) {
    using Pk = Pack<PREC, V>;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool from_wall = WALL >= 0 && q != 0 && (WALL == 0 ? cy(q) > 0 : cy(q) < 0);
        if (!ODD || from_wall) {
            pk[q].vload(base + q * np + idx0);
        } else {
            const int p = opp(q);  // read plane opp(q) at x - c_q = x + c_p
            if (cx(p) == 0) {
                pk[q].vload(base + p * np + idx0 + yz_off(cg, p));
            } else {
                // the V values straddle two aligned groups of the row: the
                // neighbour group on the side of c_p (wrapped at the row end)
                // and the group itself
                const typename Store<PREC>::T *plane = base + p * np + idx0 + yz_off(cg, p);
                Pk own, nbr;
                own.vload(plane);
                nbr.vload(plane + (cx(p) > 0 ? (cg.x + V == L.nx ? V - L.nx : V) : (cg.x == 0 ? L.nx - V : -V)));
                pk[q].shifted(cx(p) > 0, own, nbr);
            }
        }
    }
}

// Stores of a group's post-collision values (pk[q]: direction q of each
// cell): even steps slot opp(q) of the cell itself; odd steps slot q of
// x + c_q, and for WALL >= 0 the directions towards that wall layer bounced
// into slot opp(q) of the cell itself.  On odd steps the planes of directions
// with an x component land one element off the group's alignment and are
// stored element by element (each cell's neighbour wrapped at the row end).
template <int PREC, int ODD, int V, int WALL>
__device__ __forceinline__ void group_store(const LatDev &L, typename Store<PREC>::T *base, long long np, int idx0,
                                            const CellGeom &cg, const Pack<PREC, V> (&pk)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const bool to_wall = WALL >= 0 && (WALL == 0 ? cy(q) < 0 : cy(q) > 0);
        if (!ODD || to_wall) {
            pk[q].vstore(base + opp(q) * np + idx0);
        } else if (cx(q) == 0) {
            pk[q].vstore(base + q * np + idx0 + yz_off(cg, q));
        } else {
            typename Store<PREC>::T *row = base + q * np + idx0 + yz_off(cg, q);
            if constexpr (V == 4 && sizeof(typename Store<PREC>::T) <= 4) {
                // elements 1 and 2 land on an aligned pair inside the row
                // (x0 + 2, x0 + 3 going +x; x0, x0 + 1 going -x): one store
                pk[q].estore(row + x_off<V>(cg, L, q, 0), 0);
                pk[q].pstore12(row + (cx(q) > 0 ? 2 : 0));
                pk[q].estore(row + 3 + x_off<V>(cg, L, q, 3), 3);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) pk[q].estore(row + k + x_off<V>(cg, L, q, k), k);
            }
        }
    }
}

// The same stores for the cells of the group in `keep` only (bit k: cell
// idx0 + k), element by element where a cell is left out.
template <int PREC, int ODD, int V>
__device__ __forceinline__ void group_store_masked(const LatDev &L, typename Store<PREC>::T *base, long long np,
                                                   int idx0, const CellGeom &cg, const Pack<PREC, V> (&pk)[Q],
                                                   uint32_t keep) {
    constexpr uint32_t ALL = (1u << V) - 1u;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        typename Store<PREC>::T *row =
            !ODD ? base + opp(q) * np + idx0 : base + q * np + idx0 + yz_off(cg, q);
        if (keep == ALL && (!ODD || cx(q) == 0)) {
            pk[q].vstore(row);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k)
                if ((keep >> k) & 1u) pk[q].estore(row + k + (ODD ? x_off<V>(cg, L, q, k) : 0), k);
        }
    }
}

// Neighbour offsets of each cell of a group on its own (odd steps of a
// lattice whose nx is not a multiple of V, where a group may end a row or
// straddle two): element k of plane q sits at idx0 + k + nb_off(cell k, q).
template <int V> struct GroupGeom {
    CellGeom c[V];
};

template <int V>
__device__ __forceinline__ void group_geom(const LatDev &L, int idx0, GroupGeom<V> &gg) {
#pragma unroll
    for (int k = 0; k < V; ++k) gg.c[k] = cell_geom(L, idx0 + k);
}

// Odd-step loads of such a group, element by element (the rest direction
// from the cells' own slots, aligned).
template <int PREC, int V>
__device__ __forceinline__ void group_load_el(typename Store<PREC>::T *base, long long np, int idx0,
                                              const GroupGeom<V> &gg, Pack<PREC, V> (&pk)[Q]) {
    pk[0].vload(base + idx0);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int p = opp(q);  // read plane opp(q) at x - c_q = x + c_p
        const typename Store<PREC>::T *plane = base + p * np + idx0;
#pragma unroll
        for (int k = 0; k < V; ++k) pk[q].eload(plane + k + nb_off(gg.c[k], p), k);
    }
}

// Odd-step stores of such a group (slot q of x + c_q), the cells in `keep`.
template <int PREC, int V>
__device__ __forceinline__ void group_store_el(typename Store<PREC>::T *base, long long np, int idx0,
                                               const GroupGeom<V> &gg, const Pack<PREC, V> (&pk)[Q],
                                               uint32_t keep) {
    constexpr uint32_t ALL = (1u << V) - 1u;
    if (keep == ALL) {
        pk[0].vstore(base + idx0);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k)
            if ((keep >> k) & 1u) pk[0].estore(base + idx0 + k, k);
    }
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        typename Store<PREC>::T *plane = base + q * np + idx0;
#pragma unroll
        for (int k = 0; k < V; ++k)
            if ((keep >> k) & 1u) pk[q].estore(plane + k + nb_off(gg.c[k], q), k);
    }
}

// A group of V cells of the fluid row next to a moving wall layer (every cell
// flagged F_YLO, SIDE 0, or F_YHI, SIDE 1): the wall path of wall_cell on the
// packed group -- the same loads, arithmetic, rounding bits and per-cell
// momentum hand-over.
template <int PREC, int ODD, int V, int SIDE>
__device__ __forceinline__ void group_wall(const SweepArgs &a, const LatDev &L, int li, int idx0, uint32_t seed,
                                        uint32_t *tkey, typename Acc<PREC>::V *tval) {
    CellGeom cg;
    if (ODD) cg = cell_geom(L, idx0);
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    Pack<PREC, V> pk[Q];
    group_load<PREC, ODD, V, SIDE>(L, base, np, idx0, cg, pk);
    const LatPar<C> lp(L);
    const C *uw = SIDE == 0 ? lp.wlo : lp.whi;
    const C u0 = uw[0], u1 = uw[1], u2 = uw[2], rho0c = lp.rho0;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        C g[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) g[q] = pk[q].get(k);
        collide_lat<C>(g, L);
        Rnd<PREC> rnd(seed, L.c_off + idx0 + k);
        C sw[3] = {0, 0, 0};
        uint32_t mask = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (SIDE == 0 ? cy(q) < 0 : cy(q) > 0) {
                C cu = 0;
                if (cx(q)) cu += cx(q) > 0 ? u0 : -u0;
                cu += cy(q) > 0 ? u1 : -u1;
                if (cz(q)) cu += cz(q) > 0 ? u2 : -u2;
                const C dbb = C(6.0 * wq(q)) * rho0c * cu;
                pk[q].set(k, g[q] - dbb, rnd.next());
                const C sm = C(2) * g[q] - dbb;
                if (cx(q)) sw[0] += cx(q) > 0 ? sm : -sm;
                sw[1] += cy(q) > 0 ? sm : -sm;
                if (cz(q)) sw[2] += cz(q) > 0 ? sm : -sm;
                mask |= 1u << q;
            } else {
                pk[q].set(k, g[q], rnd.next());
            }
        }
        typename Acc<PREC>::V F[3];
        link_force<PREC>(L, sw, mask, F);
        tacc_add<PREC>(a, tkey, tval, KEY_WALL | ((uint32_t)li << 1) | (uint32_t)SIDE, F, 3);
    }
    group_store<PREC, ODD, V, SIDE>(L, base, np, idx0, cg, pk);
}

// The groups of a warp that are not plain bulk fluid on aligned rows (`mine`:
// this lane's group is one; fl: its flag bytes): a wall-row group (every cell
// F_YLO, or every cell F_YHI) on the packed wall path, any other group cell
// by cell, and then the warp's near-obstacle cells one per lane.  Out of line
// and called once per warp after the packed groups, so the bulk path has no
// call site to keep registers across and its packed values stay in
// registers.  Called by the whole warp.
template <int PREC, int ODD, int V>
__device__ __noinline__ void group_slow(const SweepArgs &a, const LatDev &L, int li, int idx0, bool mine, bool vec,
                                        uint32_t fl, int *list, uint32_t seed, uint32_t *tkey,
                                        typename Acc<PREC>::V *tval) {
    constexpr uint32_t REP = V == 2 ? 0x0101u : 0x01010101u;
    uint32_t deferred = 0;
    if (mine) {
        const uint32_t f0 = fl & 0xFFu;
        if (vec && fl == REP * f0 && f0 == (F_NEAR | F_YLO))
            group_wall<PREC, ODD, V, 0>(a, L, li, idx0, seed, tkey, tval);
        else if (vec && fl == REP * f0 && f0 == (F_NEAR | F_YHI))
            group_wall<PREC, ODD, V, 1>(a, L, li, idx0, seed, tkey, tval);
        else
            deferred = group_mixed<PREC, ODD, V>(a, L, li, idx0, fl, seed, tkey, tval);
    }
    if (__any_sync(0xffffffffu, deferred != 0)) near_pass<PREC, ODD, V>(a, L, li, idx0, deferred, list, seed, tkey, tval);
}

// One group on an aligned row whose cells in `keep` (bit k: cell idx0 + k)
// are bulk fluid: packed collision, vector accesses, stores for the kept
// cells only (MASKED; without it every cell is stored).  keep is every cell
// but in the split sweep, where a group may
// also hold near-obstacle cells (the near kernel updates them) or obstacle
// cells: the packed path then runs for the whole group and stores only the
// bulk cells.  A bulk cell has no obstacle neighbour, so its loads and
// arithmetic are those of an all-bulk group; the other cells' values are read
// and discarded (a cell's update writes exactly the slots it reads, so the
// near kernel still finds the near cells' slots untouched).  In dense
// suspensions most warps hold such a group, and this keeps them off the
// one-cell slow path.
template <int PREC, int ODD, int V, bool MASKED, bool AL = true>
__device__ __forceinline__ void group_bulk(const SweepArgs &a, const LatDev &L, int idx0, uint32_t seed,
                                           uint32_t keep) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Pk = Pack<PREC, V>;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    constexpr bool EL = ODD && !AL;  // element accesses at each cell's own offsets
    CellGeom cg;
    GroupGeom<V> gg;
    if (ODD && !EL) cg = cell_geom(L, idx0);
    if (EL) group_geom<V>(L, idx0, gg);
    Pk pk[Q];
    if constexpr (EL)
        group_load_el<PREC, V>(base, np, idx0, gg, pk);
    else
        group_load<PREC, ODD, V, -1>(L, base, np, idx0, cg, pk);
    if constexpr (PREC == LBM_F64) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            C g[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = pk[q].get(k);
            collide_lat<C>(g, L);
#pragma unroll
            for (int q = 0; q < Q; ++q) pk[q].set(k, g[q], 0u);
        }
    } else {
        // two cells per paired instruction
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            float2 g[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = pk[q].get2(k);
            collide2_lat(g, L);
            // a NaN among the outputs needs a NaN or infinite moment: with
            // the equilibrium base of both cells finite the BF16 form rounds
            // every value by integer adds
            const float b0 = g[0].x, b1 = g[0].y;
            const bool plain = PREC != LBM_BF16_OFFSET || (isfinite(b0) && isfinite(b1));
            Rnd<PREC> r0(seed, L.c_off + idx0 + k), r1(seed, L.c_off + idx0 + k + 1);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const uint32_t a0 = r0.next(), a1 = r1.next();
                pk[q].set2(k, g[q], a0, a1, plain);
            }
        }
    }
    if constexpr (EL) {
        // the offsets again rather than held across the collision (an opaque
        // copy of idx0 keeps the compiler from reusing the first ones)
        int i0;
        asm volatile("mov.b32 %0, %1;" : "=r"(i0) : "r"(idx0));
        group_geom<V>(L, i0, gg);
        group_store_el<PREC, V>(base, np, idx0, gg, pk, MASKED ? keep : (1u << V) - 1u);
    }
    else if constexpr (MASKED)
        group_store_masked<PREC, ODD, V>(L, base, np, idx0, cg, pk, keep);
    else
        group_store<PREC, ODD, V, -1>(L, base, np, idx0, cg, pk);
}

// Resident blocks of 256 threads per SM for the grouped sweep: 2 leaves 128
// registers per thread; with V cells per thread that is still V * 16 cells'
// loads in flight per SM partition against 24 for the one-cell sweep.
template <int PREC, int V> struct GroupBounds { static constexpr int MAXT = 256, MINB = 2; };

// SPLIT: the split sweep (near-obstacle cells left to the near kernel), a
// template parameter so that the other sweeps' code stays as it is.
template <int PREC, int ODD, bool SINGLE, int V, bool SPLIT>
__global__ void __launch_bounds__((GroupBounds<PREC, V>::MAXT), (GroupBounds<PREC, V>::MINB))
    sweep_group(const __grid_constant__ SweepArgs a) {
    pdl_enter();
    const uint32_t seed = PREC == LBM_BF16_OFFSET ? step_seed(a.tick) : 0u;
    __shared__ uint32_t tkey[256];
    __shared__ typename Acc<PREC>::V tval[256][6];
    __shared__ int nlist[GroupBounds<PREC, V>::MAXT / 32][32 * V];  // per warp: its deferred near cells
    tkey[threadIdx.x] = SLOT_EMPTY;
    constexpr uint32_t REP = V == 2 ? 0x0101u : 0x01010101u;
    const int tcells = V * (int)blockDim.x;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        if (a.pf_ahead[ODD]) prefetch_tile<PREC, ODD, SINGLE>(a, tile + a.pf_ahead[ODD], tcells);
        // uniform per block: a tile lies in one lattice
        const int li = tile_lattice<SINGLE>(a, tile);
        const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
        const int idx0 = (tile - L.tile0) * tcells + V * (int)threadIdx.x;
        const bool bulk_tile = a.tbits && !((a.tbits[tile >> 5] >> (tile & 31)) & 1u);
        // vector accesses need a whole group: on even steps (a cell's own
        // slots) any group but the ragged last one, on odd steps a group of
        // one row (nx a multiple of V); the others go cell by cell.  In a
        // batch, a lattice whose nx is not a multiple of V takes the packed
        // path on odd steps too, with its neighbour slots accessed element
        // by element at each cell's own offsets (`al` false; uniform per
        // block): in small lattices nearly every warp holds a group that
        // ends or straddles a row, and one such group would otherwise send
        // the warp down the one-cell path
        const bool al = !ODD || (L.nx & (V - 1)) == 0;
        const bool vec = idx0 + V <= L.n && (al || !SINGLE);
        // flag bytes of the V cells (byte k: cell idx0 + k); the flag planes
        // are padded to whole tiles of 256 cells with zeros, so the load
        // stays inside
        uint32_t fl = 0;
        if (!bulk_tile && idx0 < L.n) {
            const uint8_t *fp = a.flags + L.c_off + idx0;
            if constexpr (V == 2)
                fl = *reinterpret_cast<const unsigned short *>(fp);
            else
                fl = *reinterpret_cast<const unsigned int *>(fp);
        }
        bool slow = false;
        if (idx0 < L.n) {
            if constexpr (SPLIT) {
                // the packed path stores the bulk cells of a group whose other
                // cells are near-obstacle or obstacle cells (a wall-row cell
                // sends the group to the slow path)
                uint32_t keep = 0;
                bool other = false;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const uint32_t f = (fl >> (8 * k)) & 0xFFu;
                    if (f == 0) keep |= 1u << k;
                    else if (!(f & F_SOLID) && (f & (F_YLO | F_YHI))) other = true;
                }
                if (vec && !other) {
                    if (keep) {
                        if (SINGLE || al)
                            group_bulk<PREC, ODD, V, true>(a, L, idx0, seed, keep);
                        else
                            group_bulk<PREC, ODD, V, true, false>(a, L, idx0, seed, keep);
                    }
                } else {
                    slow = (fl & (REP * F_SOLID)) != REP * F_SOLID || !vec;
                }
            } else {
                if (vec && fl == 0) {
                    if (SINGLE || al)
                        group_bulk<PREC, ODD, V, false>(a, L, idx0, seed, (1u << V) - 1u);
                    else
                        group_bulk<PREC, ODD, V, false, false>(a, L, idx0, seed, (1u << V) - 1u);
                } else {
                    slow = (fl & (REP * F_SOLID)) != REP * F_SOLID || !vec;  // not wall or obstacle cells only
                }
            }
        }
        // the packed wall-row path wants aligned rows
        if (__any_sync(0xffffffffu, slow))
            group_slow<PREC, ODD, V>(a, L, li, idx0, slow, vec && al, fl, nlist[threadIdx.x >> 5], seed,
                                     &tkey[threadIdx.x], tval[threadIdx.x]);
    }
    flush_forces<PREC>(a, tkey, tval);
}

// ---------------------------------------------------------------------------
// Staged sweep.  A persistent block walks its tiles (256 consecutive cells of
// one lattice); one thread keeps S tiles in flight by issuing, per tile, 19
// bulk asynchronous copies global -> shared (cp.async.bulk, completion
// counted in bytes on an mbarrier).  Window q of a stage holds, for every
// cell of the tile, the population the sweep reads for direction q: on even
// steps plane q at the tile itself, on odd steps plane opp(q) shifted by the
// lattice offset of x - c_q -- a contiguous range, so one copy per plane,
// started on the 16-byte boundary below it.  The memory in flight per SM is
// set by the pipeline depth, not by registers.  Cells on a periodic face
// (odd steps only) read their wrapped neighbours from global memory.  The
// population arena has a guard band before and after it, so a shifted window
// at either end of the arena stays inside the allocation.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one mbarrier phase; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int PREC, int ODD, bool SINGLE>
__device__ __forceinline__ void issue_tile(const SweepArgs &a, int tile, typename Store<PREC>::T *stage,
                                           uint64_t *bar) {
    using Cfg = StageCfg<PREC>;
    using T = typename Store<PREC>::T;
    const int li = tile_lattice<SINGLE>(a, tile);
    const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
    const long long idx0 = (long long)(tile - L.tile0) * Cfg::TILE;
    const T *f = reinterpret_cast<const T *>(a.f) + L.f_off;
    mbar_expect_tx(bar, (uint32_t)(Cfg::STAGE_ELEMS * sizeof(T)));
#pragma unroll 1
    for (int q = 0; q < Q; ++q) {
        const int plane = ODD ? opp(q) : q;
        const long long start = idx0 + (ODD ? L.off[opp(q)] : 0);
        const long long aligned = start - (start & (Cfg::A - 1));
        bulk_copy_g2s(stage + q * Cfg::W, f + (long long)plane * L.npad + aligned,
                      (uint32_t)(Cfg::W * sizeof(T)), bar);
    }
    // the tile's flag bytes (flag planes are padded to whole tiles)
    bulk_copy_g2s(stage + Q * Cfg::W, a.flags + L.c_off + idx0, (uint32_t)Cfg::TILE, bar);
}

template <int PREC, int ODD>
__device__ __forceinline__ void bulk_cell_staged(const SweepArgs &a, const LatDev &L, int idx,
                                                 const typename Store<PREC>::T *stage, uint32_t seed) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Cfg = StageCfg<PREC>;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    C g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q)
        g[q] = S::ld(stage + q * Cfg::W + (ODD ? (L.off[opp(q)] & (Cfg::A - 1)) : 0) + threadIdx.x);
    collide_lat<C>(g, L);
    Rnd<PREC> rnd(seed, L.c_off + idx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            S::stg(base + opp(q) * np + idx, g[q], rnd.next());
        else
            S::stg(base + q * np + idx + L.off[q], g[q], rnd.next());
    }
}

template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_staged(const __grid_constant__ SweepArgs a) {
    pdl_enter();
    const uint32_t seed = PREC == LBM_BF16_OFFSET ? step_seed(a.tick) : 0u;
    using S = Store<PREC>;
    using T = typename S::T;
    using Cfg = StageCfg<PREC>;
    extern __shared__ __align__(128) unsigned char dsm[];
    T *stages = reinterpret_cast<T *>(dsm);
    __shared__ __align__(8) uint64_t bars[Cfg::S];
    __shared__ uint32_t tkey[256];
    __shared__ typename Acc<PREC>::V tval[256][6];
    const int tid = threadIdx.x;
    tkey[tid] = SLOT_EMPTY;
#pragma unroll
    for (int k = 0; k < 6; ++k) tval[tid][k] = Acc<PREC>::zero();
    if (tid == 0) {
        for (int s = 0; s < Cfg::S; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int nk = blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0)
        for (int k = 0; k < Cfg::S - 1 && k < nk; ++k)
            issue_tile<PREC, ODD, SINGLE>(a, blockIdx.x + k * gridDim.x, stages + k * Cfg::STAGE_ELEMS, &bars[k]);
    int issued = nk < Cfg::S - 1 ? nk : Cfg::S - 1;
    bool timed_out = false;
    for (int k = 0; k < nk; ++k) {
        if (tid == 0 && issued < nk) {
            // the stage being refilled was last read by tile k-1, which every
            // thread finished before the barrier that ended its iteration
            const int sn = issued % Cfg::S;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<PREC, ODD, SINGLE>(a, blockIdx.x + issued * gridDim.x, stages + sn * Cfg::STAGE_ELEMS,
                                          &bars[sn]);
            ++issued;
        }
        const int s = k % Cfg::S;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / Cfg::S) & 1));
        if (ok) {
            const int tile = blockIdx.x + k * gridDim.x;
            const int li = tile_lattice<SINGLE>(a, tile);
            const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
            const int idx = (tile - L.tile0) * Cfg::TILE + tid;
            const T *stage = stages + s * Cfg::STAGE_ELEMS;
            if (idx < L.n) {
                const uint8_t fl = reinterpret_cast<const uint8_t *>(stage + Q * Cfg::W)[tid];
                if (!(fl & F_SOLID)) {
                    CellGeom cg;
                    const uint32_t yz = L.divx.div((uint32_t)idx);
                    cg.x = idx - (int)yz * L.nx;
                    cg.z = (int)L.divxy.div((uint32_t)idx);
                    cg.y = (int)yz - cg.z * L.ny;
                    const bool interior = !ODD || (cg.x > 0 && cg.x < L.nx - 1 && cg.y > 0 && cg.y < L.ny - 1 &&
                                                   cg.z > 0 && cg.z < L.nz - 1);
                    if (interior && !(fl & F_NEAR)) {
                        bulk_cell_staged<PREC, ODD>(a, L, idx, stage, seed);
                    } else {
                        const int sy = L.nx, sz = L.nx * L.ny;
                        cg.dxm = cg.x == 0 ? L.nx - 1 : -1;
                        cg.dxp = cg.x == L.nx - 1 ? -(L.nx - 1) : 1;
                        cg.dym = cg.y == 0 ? (L.ny - 1) * sy : -sy;
                        cg.dyp = cg.y == L.ny - 1 ? -(L.ny - 1) * sy : sy;
                        cg.dzm = cg.z == 0 ? (L.nz - 1) * sz : -sz;
                        cg.dzp = cg.z == L.nz - 1 ? -(L.nz - 1) * sz : sz;
                        if (fl & F_NEAR) {
                            typename S::C g[Q];
                            if (interior)
                                near_cell<PREC, ODD, 1>(a, L, li, idx, &tkey[tid], tval[tid], stage, g, seed);
                            else
                                near_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[tid], tval[tid], nullptr, g, seed);
                        } else {
                            bulk_cell<PREC, ODD>(a, L, idx, seed);
                        }
                    }
                }
            }
        }
        // every thread is done with stage s; stop together if a wait ran out
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
    }
    if (timed_out) {
        if (tid == 0) {
            atomicOr(a.err, ERR_TIMEOUT);
            // let copies still in flight land before the block's shared memory
            // goes away (each wait bounded)
            for (int k2 = issued - Cfg::S; k2 < issued; ++k2)
                if (k2 >= 0) mbar_wait_bounded(&bars[k2 % Cfg::S], (uint32_t)((k2 / Cfg::S) & 1));
        }
        __syncthreads();
    }
    flush_forces<PREC>(a, tkey, tval);
}

// ---------------------------------------------------------------------------
// Ring sweep.  Every thread prefetches the populations (and the flag word) of
// the cell it will update D tiles later with asynchronous copies into its own
// column of a shared-memory ring (cp.async, 4 or 8 bytes each), and waits
// only for its own copy groups (cp.async.wait_group): the loop has no block
// barrier, and each thread keeps D+1 cells of loads in flight instead of one,
// without holding them in registers.  Addresses are the cell's own pull
// addresses (periodic wrap included), so no cell needs a separate path; on
// odd steps a near-obstacle cell re-reads from global memory the populations
// whose source neighbour is an obstacle.  In the AA pattern the slots a cell
// reads are written only by that cell, so reading them early is race-free.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the copies of one cell into this thread's ring column.
template <int PREC, int ODD>
__device__ __forceinline__ void ring_fetch(const SweepArgs &a, const LatDev &L, int idx,
                                           typename RingCfg<PREC>::Word *col) {
    using T = typename Store<PREC>::T;
    using Cfg = RingCfg<PREC>;
    const T *base = reinterpret_cast<const T *>(a.f) + L.f_off;
    const long long np = L.npad;
    CellGeom cg;
    if (ODD) cg = cell_geom(L, idx);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const T *src = ODD ? base + opp(q) * np + idx + nb_off(cg, opp(q)) : base + q * np + idx;
        if (sizeof(T) == 8)
            cp_async_8(col + q * Cfg::TILE, src);
        else if (sizeof(T) == 4)
            cp_async_4(col + q * Cfg::TILE, src);
        else
            cp_async_4(col + q * Cfg::TILE, reinterpret_cast<const void *>((uintptr_t)src & ~(uintptr_t)3));
    }
    const uint8_t *fl = a.flags + L.c_off + idx;
    cp_async_4(col + Q * Cfg::TILE, reinterpret_cast<const void *>((uintptr_t)fl & ~(uintptr_t)3));
}

template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_ring(const __grid_constant__ SweepArgs a) {
    pdl_enter();
    const uint32_t seed = PREC == LBM_BF16_OFFSET ? step_seed(a.tick) : 0u;
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Cfg = RingCfg<PREC>;
    using Word = typename Cfg::Word;
    extern __shared__ __align__(128) unsigned char dsm[];
    Word *ring = reinterpret_cast<Word *>(dsm);
    __shared__ uint32_t tkey[256];
    __shared__ typename Acc<PREC>::V tval[256][6];
    const int tid = threadIdx.x;
    tkey[tid] = SLOT_EMPTY;
#pragma unroll
    for (int k = 0; k < 6; ++k) tval[tid][k] = Acc<PREC>::zero();

    const int nk = blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // prologue: tiles 0 .. D-1 (one commit group per tile, empty groups included)
#pragma unroll
    for (int j = 0; j < Cfg::D; ++j) {
        if (j < nk) {
            const int tile = blockIdx.x + j * gridDim.x;
            const LatDev &L = SINGLE ? a.lat0 : a.lat[tile_lattice<SINGLE>(a, tile)];
            const int idx = (tile - L.tile0) * Cfg::TILE + tid;
            if (idx < L.n) ring_fetch<PREC, ODD>(a, L, idx, ring + j * Cfg::SLOT + tid);
        }
        cp_async_commit();
    }
    for (int k = 0; k < nk; ++k) {
        {
            const int kf = k + Cfg::D;
            if (kf < nk) {
                const int tile = blockIdx.x + kf * gridDim.x;
                const LatDev &L = SINGLE ? a.lat0 : a.lat[tile_lattice<SINGLE>(a, tile)];
                const int idx = (tile - L.tile0) * Cfg::TILE + tid;
                if (idx < L.n) ring_fetch<PREC, ODD>(a, L, idx, ring + (kf % (Cfg::D + 1)) * Cfg::SLOT + tid);
            }
            cp_async_commit();
        }
        cp_async_wait<Cfg::D>();  // this thread's copies of tile k have landed
        const int tile = blockIdx.x + k * gridDim.x;
        const int li = tile_lattice<SINGLE>(a, tile);
        const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
        const int idx = (tile - L.tile0) * Cfg::TILE + tid;
        if (idx >= L.n) continue;
        const Word *col = ring + (k % (Cfg::D + 1)) * Cfg::SLOT + tid;
        const uint32_t fw = (uint32_t)col[Q * Cfg::TILE];
        const uint8_t fl = (uint8_t)(fw >> (8 * (int)((L.c_off + idx) & 3)));
        if (fl & F_SOLID) continue;
        const CellGeom cg = cell_geom(L, idx);
        if (fl & F_NEAR) {
            C gn[Q];
            near_cell<PREC, ODD, 2>(a, L, li, idx, &tkey[tid], tval[tid], col, gn, seed);
            continue;
        }
        C g[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q)
            g[q] = ring_value<PREC>(col, q, ODD ? ((idx + nb_off(cg, opp(q))) & 1) : (idx & 1));
        collide_lat<C>(g, L);
        Rnd<PREC> rnd(seed, L.c_off + idx);
        T *base = reinterpret_cast<T *>(a.f) + L.f_off;
        const long long np = L.npad;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!ODD)
                S::stg(base + opp(q) * np + idx, g[q], rnd.next());
            else
                S::stg(base + q * np + idx + nb_off(cg, q), g[q], rnd.next());
        }
    }
    cp_async_wait<0>();
    flush_forces<PREC>(a, tkey, tval);
}

// Split sweep, step 1: the near-obstacle cells (F_NEAR without a flat-wall
// flag) of the tiles marked in the tile bits, compacted into a.near_list.
// Each warp takes a contiguous range of tpw tiles: it counts its cells, a
// lane reading eight flag bytes with one load, reserves its slice of the
// list with one atomic and writes the cells in tile and cell order (lane l
// holds cells 8l .. 8l+7 of each 256 of the tile), so neighbouring list
// entries are neighbouring cells.  One atomic per warp with cells rather
// than per tile (same-address atomics serialise), no barrier, and every
// load of a warp independent of the warp's other loads.
__device__ __forceinline__ bool near_listed(uint8_t fl) { return (fl & F_NEAR) && !(fl & (F_YLO | F_YHI)); }

// Bit b of the result: cell c + b of the tile is listed (c a multiple of 8;
// bytes at or beyond the lattice's last cell count as empty).
__device__ __forceinline__ uint32_t near_bits8(const uint8_t *fp, int c, int valid) {
    if (c >= valid) return 0u;
    const uint2 w = *reinterpret_cast<const uint2 *>(fp + c);
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint8_t fl = (uint8_t)((b < 4 ? w.x : w.y) >> (8 * (b & 3)));
        if (c + b < valid && near_listed(fl)) m |= 1u << b;
    }
    return m;
}

template <bool SINGLE>
__global__ void __launch_bounds__(256) near_list_kernel(const __grid_constant__ SweepArgs a, int tcells, int tpw) {
    pdl_enter();
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int t0 = warp * tpw, t1 = min(a.ntiles, t0 + tpw);
    uint32_t n = 0;  // this lane's cells
    for (int tile = t0; tile < t1; ++tile) {
        if (a.tbits && !((a.tbits[tile >> 5] >> (tile & 31)) & 1u)) continue;  // uniform per warp
        const LatDev &L = SINGLE ? a.lat0 : a.lat[tile_lattice<SINGLE>(a, tile)];
        const int s0 = (tile - L.tile0) * tcells;
        const uint8_t *fp = a.flags + L.c_off + s0;
        const int valid = min(tcells, L.n - s0);
        for (int c = 8 * lane; c < tcells; c += 256) n += (uint32_t)__popc(near_bits8(fp, c, valid));
    }
    // inclusive prefix of the lanes' counts
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    if (total == 0) return;  // the whole warp
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(a.near_count, total);
    base = __shfl_sync(FULL, base, 0);
    // second walk: per tile (and per 256 cells of it) the lanes' counts again,
    // written from the warp's running offset in cell order
    for (int tile = t0; tile < t1; ++tile) {
        if (a.tbits && !((a.tbits[tile >> 5] >> (tile & 31)) & 1u)) continue;
        const LatDev &L = SINGLE ? a.lat0 : a.lat[tile_lattice<SINGLE>(a, tile)];
        const int s0 = (tile - L.tile0) * tcells;
        const uint8_t *fp = a.flags + L.c_off + s0;
        const int valid = min(tcells, L.n - s0);
        for (int cb = 0; cb < tcells; cb += 256) {
            const int c = cb + 8 * lane;
            uint32_t m = c < tcells ? near_bits8(fp, c, valid) : 0u;
            const uint32_t cnt = (uint32_t)__popc(m);
            uint32_t x = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += v;
            }
            uint32_t pos = base + x - cnt;
            for (; m; m &= m - 1) a.near_list[pos++] = (uint32_t)(L.c_off + s0 + c + __ffs(m) - 1);
            base += __shfl_sync(FULL, x, 31);
        }
    }
}

// Split sweep, step 3: one thread per listed near-obstacle cell (a
// persistent grid over the list), the same update as the fused path.  (A
// contiguous slice of the list per warp, which would let a thread's partial
// sums run over cells of one body, measured slower on GB300 than the grid
// stride, whose concurrent warps work on neighbouring list entries.)
template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB) near_kernel(const __grid_constant__ SweepArgs a) {
    pdl_enter();
    const uint32_t seed = PREC == LBM_BF16_OFFSET ? step_seed(a.tick) : 0u;
    using C = typename Store<PREC>::C;
    __shared__ uint32_t tkey[256];
    __shared__ typename Acc<PREC>::V tval[256][6];
    tkey[threadIdx.x] = SLOT_EMPTY;
    const uint32_t n = *a.near_count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t cell = a.near_list[i];
        int li = 0;
        if (!SINGLE) {
            int lo = 0, hi = a.nlat - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.lat[mid].c_off <= (long long)cell) lo = mid; else hi = mid - 1;
            }
            li = lo;
        }
        const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
        const int idx = (int)((long long)cell - L.c_off);
        C g[Q];
        near_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x], nullptr, g, seed);
    }
    flush_forces<PREC>(a, tkey, tval);
}

// Host-side per-device state of the launchers: whether the dynamic shared
// memory attribute of a kernel has been raised on a device, and the resident
// blocks of the near kernel over all of a device's SMs.  Keyed by device and
// guarded by one mutex (launches come from any host thread, each context on
// its own device).
constexpr int LAUNCH_MAX_DEVICES = 64;
inline std::mutex &launch_cache_mu() {
    static std::mutex m;
    return m;
}

template <class K>
cudaError_t raise_smem_once(K kernel, int smem, bool (&done)[LAUNCH_MAX_DEVICES]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= LAUNCH_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(launch_cache_mu());
    if (!done[dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

template <int PREC, int ODD, bool SINGLE>
cudaError_t launch_direct(const SweepArgs &a, int grid, int block, int cpt, cudaStream_t s) {
    const bool split = a.near_list != nullptr;
    if (cpt == 2)
        return split ? launch_pdl(sweep_group<PREC, ODD, SINGLE, 2, true>, grid, block, 0, s, a)
                     : launch_pdl(sweep_group<PREC, ODD, SINGLE, 2, false>, grid, block, 0, s, a);
    if constexpr (PREC != LBM_F64) {
        if (cpt == 4)
            return split ? launch_pdl(sweep_group<PREC, ODD, SINGLE, 4, true>, grid, block, 0, s, a)
                         : launch_pdl(sweep_group<PREC, ODD, SINGLE, 4, false>, grid, block, 0, s, a);
    }
    if (cpt != 1) return cudaErrorInvalidValue;
    return launch_pdl(sweep_kernel<PREC, ODD, SINGLE>, grid, block, 0, s, a);
}

template <int PREC, int ODD, bool SINGLE>
cudaError_t launch_one(int variant, const SweepArgs &a, int grid, int block, int cpt, cudaStream_t s) {
    if (variant == SWEEP_STAGED) {
        constexpr int smem = StageCfg<PREC>::SMEM;
        static bool attr[LAUNCH_MAX_DEVICES] = {};
        cudaError_t e = raise_smem_once(sweep_staged<PREC, ODD, SINGLE>, smem, attr);
        if (e != cudaSuccess) return e;
        return launch_pdl(sweep_staged<PREC, ODD, SINGLE>, grid, StageCfg<PREC>::TILE, smem, s, a);
    } else if (variant == SWEEP_RING) {
        constexpr int smem = RingCfg<PREC>::SMEM;
        static bool attr[LAUNCH_MAX_DEVICES] = {};
        cudaError_t e = raise_smem_once(sweep_ring<PREC, ODD, SINGLE>, smem, attr);
        if (e != cudaSuccess) return e;
        return launch_pdl(sweep_ring<PREC, ODD, SINGLE>, grid, RingCfg<PREC>::TILE, smem, s, a);
    } else if (a.near_list) {
        static int wave[LAUNCH_MAX_DEVICES] = {};  // resident near-kernel blocks on all SMs, per device
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= LAUNCH_MAX_DEVICES) return cudaErrorInvalidDevice;
        int nwave;
        {
            std::lock_guard<std::mutex> lock(launch_cache_mu());
            if (!wave[dev]) {
                int sms = 0, nb = 0;
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, near_kernel<PREC, ODD, SINGLE>, 128, 0);
                wave[dev] = (sms > 0 ? sms : 1) * (nb > 0 ? nb : 1);
            }
            nwave = wave[dev];
        }
        e = cudaMemsetAsync(a.near_count, 0, sizeof(uint32_t), s);
        // tiles per list warp: about 48 warps per SM over all tiles
        const int tcells = block * cpt;
        const int want = nwave * 4;
        const int tpw = a.ntiles > want ? (a.ntiles + want - 1) / want : 1;
        const int lwarps = (a.ntiles + tpw - 1) / tpw;
        if (e == cudaSuccess) e = launch_pdl(near_list_kernel<SINGLE>, (lwarps + 7) / 8, 256, 0, s, a, tcells, tpw);
        if (e == cudaSuccess) e = launch_direct<PREC, ODD, SINGLE>(a, grid, block, cpt, s);
        if (e == cudaSuccess) e = launch_pdl(near_kernel<PREC, ODD, SINGLE>, nwave, 128, 0, s, a);
        return e;
    } else {
        return launch_direct<PREC, ODD, SINGLE>(a, grid, block, cpt, s);
    }
}

}  // namespace

template <int PREC>
cudaError_t launch_sweep_prec(int parity, int variant, const SweepArgs &a, int grid, int block, int cpt,
                              cudaStream_t s) {
    const bool single = a.nlat == 1;
    if (parity)
        return single ? launch_one<PREC, 1, true>(variant, a, grid, block, cpt, s)
                      : launch_one<PREC, 1, false>(variant, a, grid, block, cpt, s);
    return single ? launch_one<PREC, 0, true>(variant, a, grid, block, cpt, s)
                  : launch_one<PREC, 0, false>(variant, a, grid, block, cpt, s);
}

template <int PREC>
int sweep_max_blocks_prec(int variant, int block, int cpt) {
    int nb = 0;
    if (variant == SWEEP_STAGED) {
        constexpr int smem = StageCfg<PREC>::SMEM;
        cudaFuncSetAttribute(sweep_staged<PREC, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_staged<PREC, 1, false>, StageCfg<PREC>::TILE,
                                                      smem);
    } else if (variant == SWEEP_RING) {
        constexpr int smem = RingCfg<PREC>::SMEM;
        cudaFuncSetAttribute(sweep_ring<PREC, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_ring<PREC, 1, false>, RingCfg<PREC>::TILE, smem);
    } else if (cpt == 2) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_group<PREC, 1, false, 2, false>, block, 0);
    } else if (cpt == 4) {
        if constexpr (PREC != LBM_F64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_group<PREC, 1, false, 4, false>, block, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<PREC, 1, false>, block, 0);
    }
    return nb;
}

}  // namespace lbm
