// lbm_sweep.cu -- the fused stream-collide sweep (Sec. 4.1, Eqs. LBMCollide and
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
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr int NSLOT = 32;
constexpr uint32_t SLOT_EMPTY = 0xFFFFFFFFu;
constexpr uint32_t KEY_WALL = 0x80000000u;

// Lattice tables for runtime-indexed use in the bounce-back helper.
__constant__ int c_cx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__constant__ int c_cy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__constant__ int c_cz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__constant__ double c_w[Q] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
                              1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
                              1.0 / 36.0};

// Shared memory of a sweep block: a small hash table of per-body partial
// sums, and one partial-sum entry per thread.
struct Slots {
    uint32_t key[NSLOT];
    double v[NSLOT][6];
};

__device__ __forceinline__ double *global_acc(const SweepArgs &a, uint32_t key) {
    const size_t c = (blockIdx.x * 8u + (threadIdx.x >> 5)) & (ACC_COPIES - 1);
    if (key & KEY_WALL) {
        const size_t l = (key & ~KEY_WALL) >> 1;
        return a.wall_acc + 6 * (l * ACC_COPIES + c) + 3 * (key & 1u);
    }
    return a.P.acc + 6 * ((size_t)key * ACC_COPIES + c);
}

// Add a partial sum to the block table (or straight to global memory when
// the table is full).  Wall keys carry only a force.
__device__ void slot_add(Slots *sh, const SweepArgs &a, uint32_t key, const double *v) {
    const int nv = (key & KEY_WALL) ? 3 : 6;
    const uint32_t h = (key * 2654435761u) % NSLOT;
    for (int i = 0; i < NSLOT; ++i) {
        const uint32_t s = (h + i) % NSLOT;
        const uint32_t old = atomicCAS(&sh->key[s], SLOT_EMPTY, key);
        if (old == SLOT_EMPTY || old == key) {
            for (int k = 0; k < nv; ++k) atomicAdd(&sh->v[s][k], v[k]);
            return;
        }
    }
    double *g = global_acc(a, key);
    for (int k = 0; k < nv; ++k) atomicAdd(g + k, v[k]);
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
// enters as the odd source 3 w rho0 c.g.
template <class C>
__device__ __forceinline__ void collide(C (&g)[Q], C om, C oo, C rho0, C gx, C gy, C gz) {
    C dr = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        dr += g[q];
        if (cx(q)) jx += cx(q) > 0 ? g[q] : -g[q];
        if (cy(q)) jy += cy(q) > 0 ? g[q] : -g[q];
        if (cz(q)) jz += cz(q) > 0 ? g[q] : -g[q];
    }
    const C inv = C(1) / rho0;
    const C ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const C base = dr - C(1.5) * rho0 * (ux * ux + uy * uy + uz * uz);
    g[0] = g[0] - om * (g[0] - C(wq(0)) * base);
#pragma unroll
    for (int q = 1; q < Q; q += 2) {
        const C w = C(wq(q));
        C cu = 0, cg = 0;
        if (cx(q)) { cu += cx(q) > 0 ? ux : -ux; cg += cx(q) > 0 ? gx : -gx; }
        if (cy(q)) { cu += cy(q) > 0 ? uy : -uy; cg += cy(q) > 0 ? gy : -gy; }
        if (cz(q)) { cu += cz(q) > 0 ? uz : -uz; cg += cz(q) > 0 ? gz : -gz; }
        const C ge = C(0.5) * (g[q] + g[q + 1]);
        const C go = C(0.5) * (g[q] - g[q + 1]);
        const C feq_e = w * (base + C(4.5) * rho0 * cu * cu);
        const C feq_o = C(3) * w * rho0 * cu;
        const C ne = om * (ge - feq_e);
        const C no = oo * (go - feq_o) - C(3) * w * rho0 * cg;
        g[q] = g[q] - ne - no;
        g[q + 1] = g[q + 1] - ne + no;
    }
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
    int lo = 0, hi = a.nlat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Add nv components to this thread's partial sum for `key` (a body or a
// wall).  A thread holds one key at a time; meeting another key first hands
// the held partial to the global accumulators.
__device__ __forceinline__ void tacc_add(const SweepArgs &a, uint32_t *tkey, double *tval, uint32_t key,
                                         const double *v, int nv) {
    if (*tkey != key) {
        if (*tkey != SLOT_EMPTY) {
            double *g = global_acc(a, *tkey);
            const int nk = (*tkey & KEY_WALL) ? 3 : 6;
            for (int k = 0; k < nk; ++k) atomicAdd(g + k, tval[k]);
        }
        *tkey = key;
        for (int k = 0; k < 6; ++k) tval[k] = 0.0;
    }
    for (int k = 0; k < nv; ++k) tval[k] += v[k];
}

// Velocity bounce-back of one link (Eq. LBMMovWall) and its momentum
// exchange (Eqs. TransferredMomentum, LBMhydrodynForce).  ft is the
// post-collision offset f~_q - w_q rho0 of the fluid cell; returns the offset
// of the reflected population f~_q - 6 w_q rho0 c_q.u_s.  The momentum
// (2 f~_q - 6 w_q rho0 c_q.u_s) c_q, and its torque (x_s - x_C) x dF about the
// body centre, go into this thread's partial-sum entry.
__device__ __noinline__ double bounce_link(const SweepArgs &a, const LatDev &L, int li, int q, int nb,
                                           int xs, int ys, int zs, double ft, uint32_t *tkey,
                                           double *tval, Slots *sh) {
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
        tacc_add(a, tkey, tval, key, v, 6);
    }
    return ft - dbb;
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
// 1 the bulk-copy stage window `src`, 2 the thread's ring column `src`; the
// populations bounced off obstacles in the previous step always come from
// global memory.
// Only scalars and pointers cross the call, so the caller's register arrays
// never need an address (which would put them in local memory on every path).
template <int PREC, int ODD, int VIEW>
__device__ __noinline__ void near_cell(const SweepArgs &a, const LatDev &L, int li, int idx,
                                       uint32_t *tkey, double *tval, Slots *sh, const void *src) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Cfg = StageCfg<PREC>;
    const CellGeom cg = cell_geom(L, idx);
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    const T *stage = reinterpret_cast<const T *>(src);
    const typename RingCfg<PREC>::Word *col = reinterpret_cast<const typename RingCfg<PREC>::Word *>(src);
    uint32_t solid = 0;  // bit q: x + c_q is a wall or obstacle cell
    uint32_t wall = 0;   // bit q: x + c_q is a wall-layer cell
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const uint8_t f = a.flags[L.c_off + idx + nb_off(cg, q)];
        if (f & F_SOLID) solid |= 1u << q;
        if (f & F_WALL) wall |= 1u << q;
    }
    C g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int p = opp(q);
        if (!ODD) {
            if (VIEW == 1) g[q] = S::ld(stage + q * Cfg::W + threadIdx.x);
            else if (VIEW == 2) g[q] = ring_value<PREC>(col, q, idx & 1);
            else if (VIEW == 3) g[q] = reinterpret_cast<const C *>(src)[q];
            else g[q] = S::ld(base + q * np + idx);
        } else if ((solid >> p) & 1u) {
            g[q] = S::ld(base + q * np + idx);
        } else if (VIEW == 3) {
            g[q] = reinterpret_cast<const C *>(src)[q];
        } else if (VIEW == 1) {
            g[q] = S::ld(stage + q * Cfg::W + (L.off[p] & (Cfg::A - 1)) + threadIdx.x);
        } else if (VIEW == 2) {
            g[q] = ring_value<PREC>(col, q, (idx + nb_off(cg, p)) & 1);
        } else {
            g[q] = S::ld(base + p * np + idx + nb_off(cg, p));
        }
    }
    // Obstacle links: the ids of all obstacle neighbours are requested in one
    // round trip; the first body met (p0) has its state loaded once and its
    // links are bounced inline, in FP64, with the force and torque summed in
    // registers; links to any further body take bounce_link.
    const uint32_t obst = solid & ~wall;
    uint32_t p0 = SLOT_EMPTY, m0 = 0;
    if (obst) {
        uint32_t ids[Q];
#pragma unroll
        for (int q = 1; q < Q; ++q)
            ids[q] = ((obst >> q) & 1u) ? a.pid[L.c_off + idx + nb_off(cg, q)] : SLOT_EMPTY;
#pragma unroll
        for (int q = 1; q < Q; ++q)
            if (ids[q] != SLOT_EMPTY) {
                if (p0 == SLOT_EMPTY) p0 = ids[q];
                if (ids[q] == p0) m0 |= 1u << q;
            }
    }
    double bpos[3] = {0, 0, 0}, bU[3] = {0, 0, 0}, bW[3] = {0, 0, 0};
    if (p0 != SLOT_EMPTY) {
        for (int k = 0; k < 3; ++k) {
            bpos[k] = a.P.pos[3 * (size_t)p0 + k];
            bU[k] = a.P.vel[3 * (size_t)p0 + k];
            bW[k] = a.P.om[3 * (size_t)p0 + k];
        }
    }
    double bacc[6] = {0, 0, 0, 0, 0, 0};
    collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
    // Wall links are bounced inline in the compute precision: the wall layer
    // that is hit follows from the neighbour's y (a y = 0 or y = ny-1 layer
    // of a non-periodic y axis moves, any other wall layer rests).  Their
    // momentum is summed per cell as a small part (2 f~ - 6 w rho0 c.u_w, with
    // f~ the stored offset) and the constant part 2 w rho0 c, then handed to
    // the FP64 per-thread partial once.  Obstacle (particle) links go through
    // bounce_link in FP64.
    C wsmall[3] = {0, 0, 0}, wconst[3] = {0, 0, 0};
    int wside = -1;
    const C rho0c = C(L.rho0);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if ((wall >> q) & 1u) {
            const int ys = cg.y + cy(q);
            int side = -1;
            C u0 = 0, u1 = 0, u2 = 0;
            if (!L.py && ys == 0) {
                side = 0;
                u0 = C(L.wlo[0]); u1 = C(L.wlo[1]); u2 = C(L.wlo[2]);
            } else if (!L.py && ys == L.ny - 1) {
                side = 1;
                u0 = C(L.whi[0]); u1 = C(L.whi[1]); u2 = C(L.whi[2]);
            }
            C cu = 0;
            if (cx(q)) cu += cx(q) > 0 ? u0 : -u0;
            if (cy(q)) cu += cy(q) > 0 ? u1 : -u1;
            if (cz(q)) cu += cz(q) > 0 ? u2 : -u2;
            const C dbb = C(6.0 * wq(q)) * rho0c * cu;
            const C val = g[q] - dbb;
            if (side >= 0) {
                if (wside >= 0 && side != wside) {  // a cell touching both y walls (ny = 3): flush first
                    double v[6] = {(double)wsmall[0] + (double)wconst[0], (double)wsmall[1] + (double)wconst[1],
                                   (double)wsmall[2] + (double)wconst[2], 0, 0, 0};
                    double *gacc = global_acc(a, KEY_WALL | ((uint32_t)li << 1) | (uint32_t)wside);
                    for (int k = 0; k < 3; ++k) atomicAdd(gacc + k, v[k]);
                    wsmall[0] = wsmall[1] = wsmall[2] = wconst[0] = wconst[1] = wconst[2] = 0;
                }
                wside = side;
                const C ms = C(2) * g[q] - dbb, mc = C(2.0 * wq(q)) * rho0c;
                if (cx(q)) { wsmall[0] += cx(q) > 0 ? ms : -ms; wconst[0] += cx(q) > 0 ? mc : -mc; }
                if (cy(q)) { wsmall[1] += cy(q) > 0 ? ms : -ms; wconst[1] += cy(q) > 0 ? mc : -mc; }
                if (cz(q)) { wsmall[2] += cz(q) > 0 ? ms : -ms; wconst[2] += cz(q) > 0 ? mc : -mc; }
            }
            S::st(base + opp(q) * np + idx, val);
        } else if ((m0 >> q) & 1u) {
            // velocity bounce-back off body p0 (Eq. LBMMovWall) and the link's
            // momentum (2 f~ - 6 w rho0 c.u_s) c and torque (x_s - x_C) x dF
            const double r0 = min_image((double)wrapc(cg.x + cx(q), L.nx) - bpos[0], L.nx, L.px);
            const double r1 = min_image((double)wrapc(cg.y + cy(q), L.ny) - bpos[1], L.ny, L.py);
            const double r2 = min_image((double)wrapc(cg.z + cz(q), L.nz) - bpos[2], L.nz, L.pz);
            const double us0 = bU[0] + (bW[1] * r2 - bW[2] * r1);
            const double us1 = bU[1] + (bW[2] * r0 - bW[0] * r2);
            const double us2 = bU[2] + (bW[0] * r1 - bW[1] * r0);
            const double cu = cx(q) * us0 + cy(q) * us1 + cz(q) * us2;
            const double dbb = 6.0 * wq(q) * L.rho0 * cu;
            const double ft = (double)g[q];
            S::st(base + opp(q) * np + idx, (C)(ft - dbb));
            const double mag = 2.0 * (ft + wq(q) * L.rho0) - dbb;
            const double f0 = mag * cx(q), f1 = mag * cy(q), f2 = mag * cz(q);
            bacc[0] += f0;
            bacc[1] += f1;
            bacc[2] += f2;
            bacc[3] += r1 * f2 - r2 * f1;
            bacc[4] += r2 * f0 - r0 * f2;
            bacc[5] += r0 * f1 - r1 * f0;
        } else if ((solid >> q) & 1u) {
            const double v = bounce_link(a, L, li, q, idx + nb_off(cg, q), wrapc(cg.x + cx(q), L.nx),
                                         wrapc(cg.y + cy(q), L.ny), wrapc(cg.z + cz(q), L.nz),
                                         (double)g[q], tkey, tval, sh);
            S::st(base + opp(q) * np + idx, (C)v);
        } else if (!ODD) {
            S::st(base + opp(q) * np + idx, g[q]);
        } else {
            S::st(base + q * np + idx + nb_off(cg, q), g[q]);
        }
    }
    if (p0 != SLOT_EMPTY) tacc_add(a, tkey, tval, p0, bacc, 6);
    if (wside >= 0) {
        const uint32_t key = KEY_WALL | ((uint32_t)li << 1) | (uint32_t)wside;
        double v[3];
        for (int k = 0; k < 3; ++k) v[k] = (double)wsmall[k] + (double)wconst[k];
        tacc_add(a, tkey, tval, key, v, 3);
    }
}

// Fluid cell whose only wall/obstacle neighbours are the moving wall layer
// y = 0 (SIDE 0) or y = ny-1 (SIDE 1): the bounced directions are the five with
// c_y = -1 (resp. +1), known at compile time, so the whole update stays in the
// bulk path's registers.  On odd steps the five populations arriving from the
// layer are the ones the previous step bounced into slot q of x itself.
template <int PREC, int ODD, int SIDE>
__device__ __noinline__ void wall_cell(const SweepArgs &a, const LatDev &L, int li, int idx,
                                          uint32_t *tkey, double *tval) {
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
            g[q] = (q != 0 && (SIDE == 0 ? cy(q) > 0 : cy(q) < 0)) ? S::ld(base + q * np + idx)
                                                                  : S::ld(base + opp(q) * np + idx + nb_off(cg, opp(q)));
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) g[q] = S::ld(base + q * np + idx);
    }
    collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
    const double *uw = SIDE == 0 ? L.wlo : L.whi;
    const C u0 = C(uw[0]), u1 = C(uw[1]), u2 = C(uw[2]), rho0c = C(L.rho0);
    C ws[3] = {0, 0, 0}, wc[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (SIDE == 0 ? cy(q) < 0 : cy(q) > 0) {
            C cu = 0;
            if (cx(q)) cu += cx(q) > 0 ? u0 : -u0;
            cu += cy(q) > 0 ? u1 : -u1;
            if (cz(q)) cu += cz(q) > 0 ? u2 : -u2;
            const C dbb = C(6.0 * wq(q)) * rho0c * cu;
            S::st(base + opp(q) * np + idx, g[q] - dbb);
            const C ms = C(2) * g[q] - dbb, mc = C(2.0 * wq(q)) * rho0c;
            if (cx(q)) { ws[0] += cx(q) > 0 ? ms : -ms; wc[0] += cx(q) > 0 ? mc : -mc; }
            ws[1] += cy(q) > 0 ? ms : -ms;
            wc[1] += cy(q) > 0 ? mc : -mc;
            if (cz(q)) { ws[2] += cz(q) > 0 ? ms : -ms; wc[2] += cz(q) > 0 ? mc : -mc; }
        } else if (!ODD) {
            S::st(base + opp(q) * np + idx, g[q]);
        } else {
            S::st(base + q * np + idx + nb_off(cg, q), g[q]);
        }
    }
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = (double)ws[k] + (double)wc[k];
    tacc_add(a, tkey, tval, KEY_WALL | ((uint32_t)li << 1) | (uint32_t)SIDE, v, 3);
}

// Fluid cell with fluid neighbours only.
template <int PREC, int ODD>
__device__ __forceinline__ void bulk_cell(const SweepArgs &a, const LatDev &L, int idx, const CellGeom &cg) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    C g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            g[q] = S::ld(base + q * np + idx);
        else
            g[q] = S::ld(base + opp(q) * np + idx + nb_off(cg, opp(q)));
    }
    collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            S::st(base + opp(q) * np + idx, g[q]);
        else
            S::st(base + q * np + idx + nb_off(cg, q), g[q]);
    }
}

// Minimum resident blocks of 256 threads per SM: 3 leaves 80 registers per
// thread, enough for the bulk path to keep all 19 populations and their
// addresses in registers without spilling.
template <int PREC> struct SweepBounds { static constexpr int MINB = 3; };
template <> struct SweepBounds<LBM_F64> { static constexpr int MINB = 2; };

// SINGLE: one lattice, whose parameters travel in the kernel's parameter
// space (a.lat0) and are read as constant-bank operands; otherwise each tile
// finds its lattice in the global table by binary search on tile0.
// Hand the per-thread partial sums to the global accumulators, warp by warp:
// lanes holding the same key (body or wall) are summed by the lowest of them,
// which issues one FP64 atomic per component.  No block barrier, so blocks
// without wall or obstacle links never wait on each other's warps.
__device__ __forceinline__ void flush_forces(const SweepArgs &a, Slots &, uint32_t *tkey,
                                             double (*tval)[6]) {
    __syncwarp();
    const uint32_t key = tkey[threadIdx.x];
    const uint32_t grp = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    if (key != SLOT_EMPTY && lane == __ffs(grp) - 1) {
        double v[6] = {0, 0, 0, 0, 0, 0};
        const int wbase = threadIdx.x - lane;
        for (uint32_t m = grp; m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            for (int k = 0; k < 6; ++k) v[k] += tval[wbase + l][k];
        }
        double *g = global_acc(a, key);
        const int nv = (key & KEY_WALL) ? 3 : 6;
        for (int k = 0; k < nv; ++k) atomicAdd(g + k, v[k]);
    }
}

// Direct sweep, one cell per thread: plain stream-collide for bulk cells,
// the wall and near-obstacle paths for cells flagged F_YLO/F_YHI or F_NEAR.
template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_kernel(const __grid_constant__ SweepArgs a) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    __shared__ Slots sh;
    __shared__ uint32_t tkey[256];
    __shared__ double tval[256][6];
    tkey[threadIdx.x] = SLOT_EMPTY;

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
        const int li = tile_lattice<SINGLE>(a, tile);
        const LatDev &L = SINGLE ? a.lat0 : a.lat[li];
        const int idx = (tile - L.tile0) * blockDim.x + threadIdx.x;
        if (idx >= L.n) continue;
        T *base = reinterpret_cast<T *>(a.f) + L.f_off;
        const long long np = L.npad;
        // the 19 populations are read at the bulk pull addresses, which are in
        // range for every cell, in the same round trip as the flag byte
        C g[Q];
        CellGeom cg;
        if (ODD) {
            cg = cell_geom(L, idx);
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = S::ld(base + opp(q) * np + idx + nb_off(cg, opp(q)));
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) g[q] = S::ld(base + q * np + idx);
        }
        const uint8_t fl = a.flags[L.c_off + idx];
        if (fl & F_SOLID) continue;
        if (fl & (F_YLO | F_YHI)) {
            if (fl & F_YLO)
                wall_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x]);
            else
                wall_cell<PREC, ODD, 1>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x]);
            continue;
        }
        if (fl & F_NEAR) {  // reload from global memory inside the near path
            near_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[threadIdx.x], tval[threadIdx.x], &sh, nullptr);
            continue;
        }
        collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!ODD)
                S::st(base + opp(q) * np + idx, g[q]);
            else
                S::st(base + q * np + idx + nb_off(cg, q), g[q]);
        }
    }
    flush_forces(a, sh, tkey, tval);
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
    int li = 0;
    if (!SINGLE) {
        int lo = 0, hi = a.nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
        }
        li = lo;
    }
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
                                                 const typename Store<PREC>::T *stage) {
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
    collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (!ODD)
            S::st(base + opp(q) * np + idx, g[q]);
        else
            S::st(base + q * np + idx + L.off[q], g[q]);
    }
}

template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_staged(const __grid_constant__ SweepArgs a) {
    using S = Store<PREC>;
    using T = typename S::T;
    using Cfg = StageCfg<PREC>;
    extern __shared__ __align__(128) unsigned char dsm[];
    T *stages = reinterpret_cast<T *>(dsm);
    __shared__ __align__(8) uint64_t bars[Cfg::S];
    __shared__ Slots sh;
    __shared__ uint32_t tkey[256];
    __shared__ double tval[256][6];
    const int tid = threadIdx.x;
    tkey[tid] = SLOT_EMPTY;
#pragma unroll
    for (int k = 0; k < 6; ++k) tval[tid][k] = 0.0;
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
            int li = 0;
            if (!SINGLE) {
                int lo = 0, hi = a.nlat - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
                }
                li = lo;
            }
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
                        bulk_cell_staged<PREC, ODD>(a, L, idx, stage);
                    } else {
                        const int sy = L.nx, sz = L.nx * L.ny;
                        cg.dxm = cg.x == 0 ? L.nx - 1 : -1;
                        cg.dxp = cg.x == L.nx - 1 ? -(L.nx - 1) : 1;
                        cg.dym = cg.y == 0 ? (L.ny - 1) * sy : -sy;
                        cg.dyp = cg.y == L.ny - 1 ? -(L.ny - 1) * sy : sy;
                        cg.dzm = cg.z == 0 ? (L.nz - 1) * sz : -sz;
                        cg.dzp = cg.z == L.nz - 1 ? -(L.nz - 1) * sz : sz;
                        if (fl & F_NEAR) {
                            if (interior)
                                near_cell<PREC, ODD, 1>(a, L, li, idx, &tkey[tid], tval[tid], &sh, stage);
                            else
                                near_cell<PREC, ODD, 0>(a, L, li, idx, &tkey[tid], tval[tid], &sh, nullptr);
                        } else {
                            bulk_cell<PREC, ODD>(a, L, idx, cg);
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
    flush_forces(a, sh, tkey, tval);
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
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    using Cfg = RingCfg<PREC>;
    using Word = typename Cfg::Word;
    extern __shared__ __align__(128) unsigned char dsm[];
    Word *ring = reinterpret_cast<Word *>(dsm);
    __shared__ Slots sh;
    __shared__ uint32_t tkey[256];
    __shared__ double tval[256][6];
    const int tid = threadIdx.x;
    tkey[tid] = SLOT_EMPTY;
#pragma unroll
    for (int k = 0; k < 6; ++k) tval[tid][k] = 0.0;

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
            near_cell<PREC, ODD, 2>(a, L, li, idx, &tkey[tid], tval[tid], &sh, col);
            continue;
        }
        C g[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q)
            g[q] = ring_value<PREC>(col, q, ODD ? ((idx + nb_off(cg, opp(q))) & 1) : (idx & 1));
        collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
        T *base = reinterpret_cast<T *>(a.f) + L.f_off;
        const long long np = L.npad;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!ODD)
                S::st(base + opp(q) * np + idx, g[q]);
            else
                S::st(base + q * np + idx + nb_off(cg, q), g[q]);
        }
    }
    cp_async_wait<0>();
    flush_forces(a, sh, tkey, tval);
}

// variant: SWEEP_DIRECT (one cell per thread, `block` threads), SWEEP_STAGED
// (bulk-copy pipeline), SWEEP_RING (per-thread cp.async prefetch ring).
template <int PREC, int ODD, bool SINGLE>
cudaError_t launch_one(int variant, const SweepArgs &a, int grid, int block, cudaStream_t s) {
    if (variant == SWEEP_STAGED) {
        constexpr int smem = StageCfg<PREC>::SMEM;
        static bool attr = false;  // host-side, once per instantiation
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(sweep_staged<PREC, ODD, SINGLE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        sweep_staged<PREC, ODD, SINGLE><<<grid, StageCfg<PREC>::TILE, smem, s>>>(a);
    } else if (variant == SWEEP_RING) {
        constexpr int smem = RingCfg<PREC>::SMEM;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(sweep_ring<PREC, ODD, SINGLE>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        sweep_ring<PREC, ODD, SINGLE><<<grid, RingCfg<PREC>::TILE, smem, s>>>(a);
    } else {
        sweep_kernel<PREC, ODD, SINGLE><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_prec(int parity, int variant, const SweepArgs &a, int grid, int block, cudaStream_t s) {
    const bool single = a.nlat == 1;
    if (parity)
        return single ? launch_one<PREC, 1, true>(variant, a, grid, block, s)
                      : launch_one<PREC, 1, false>(variant, a, grid, block, s);
    return single ? launch_one<PREC, 0, true>(variant, a, grid, block, s)
                  : launch_one<PREC, 0, false>(variant, a, grid, block, s);
}

template <int PREC>
int max_blocks_prec(int variant, int block) {
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
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<PREC, 1, false>, block, 0);
    }
    return nb;
}

}  // namespace

cudaError_t launch_sweep(int prec, int parity, int variant, const SweepArgs &a, int grid, int block,
                         cudaStream_t s) {
    switch (prec) {
    case LBM_F64: return launch_prec<LBM_F64>(parity, variant, a, grid, block, s);
    case LBM_F32: return launch_prec<LBM_F32>(parity, variant, a, grid, block, s);
    case LBM_F16_OFFSET: return launch_prec<LBM_F16_OFFSET>(parity, variant, a, grid, block, s);
    case LBM_BF16_OFFSET: return launch_prec<LBM_BF16_OFFSET>(parity, variant, a, grid, block, s);
    }
    return cudaErrorInvalidValue;
}

int sweep_max_active_blocks(int prec, int variant, int block) {
    switch (prec) {
    case LBM_F64: return max_blocks_prec<LBM_F64>(variant, block);
    case LBM_F32: return max_blocks_prec<LBM_F32>(variant, block);
    case LBM_F16_OFFSET: return max_blocks_prec<LBM_F16_OFFSET>(variant, block);
    case LBM_BF16_OFFSET: return max_blocks_prec<LBM_BF16_OFFSET>(variant, block);
    }
    return 0;
}

}  // namespace lbm
