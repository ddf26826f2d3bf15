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
    if (key & KEY_WALL) {
        uint32_t l = (key & ~KEY_WALL) >> 1;
        return a.wall_acc + 6 * (size_t)l + 3 * (key & 1u);
    }
    return a.P.acc + 6 * (size_t)key;
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
        if (*tkey == SLOT_EMPTY) *tkey = key;
        if (*tkey == key) {
            for (int k = 0; k < 6; ++k) tval[k] += v[k];
        } else {
            slot_add(sh, a, key, v);
        }
    }
    return ft - dbb;
}

// Fluid cell next to walls or obstacles: neighbour flags decide where each
// population is read from (odd steps) and which outgoing populations are
// bounced back.
template <int PREC, int ODD>
__device__ __noinline__ void near_cell(const SweepArgs &a, const LatDev &L, int li, int idx,
                                       const CellGeom &cg, uint32_t *tkey, double *tval, Slots *sh) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    uint32_t solid = 0;  // bit q: x + c_q is a wall or obstacle cell
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if (a.flags[L.c_off + idx + nb_off(cg, q)] & F_SOLID) solid |= 1u << q;
    C g[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int p = opp(q);
        if (!ODD || ((solid >> p) & 1u))
            g[q] = S::ld(base + q * np + idx);
        else
            g[q] = S::ld(base + p * np + idx + nb_off(cg, p));
    }
    collide<C>(g, C(L.omega), C(L.omega_odd), C(L.rho0), C(L.g[0]), C(L.g[1]), C(L.g[2]));
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if ((solid >> q) & 1u) {
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
template <int PREC, int ODD, bool SINGLE>
__global__ void __launch_bounds__(256, SweepBounds<PREC>::MINB)
    sweep_kernel(const __grid_constant__ SweepArgs a) {
    __shared__ Slots sh;
    __shared__ uint32_t tkey[256];
    __shared__ double tval[256][6];
    for (int i = threadIdx.x; i < NSLOT; i += blockDim.x) {
        sh.key[i] = SLOT_EMPTY;
#pragma unroll
        for (int k = 0; k < 6; ++k) sh.v[i][k] = 0.0;
    }
    tkey[threadIdx.x] = SLOT_EMPTY;
#pragma unroll
    for (int k = 0; k < 6; ++k) tval[threadIdx.x][k] = 0.0;
    __syncthreads();

    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
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
        const int idx = (tile - L.tile0) * blockDim.x + threadIdx.x;
        if (idx >= L.n) continue;
        const uint8_t fl = a.flags[L.c_off + idx];
        if (fl & F_SOLID) continue;
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
        if (fl & F_NEAR)
            near_cell<PREC, ODD>(a, L, li, idx, cg, &tkey[threadIdx.x], tval[threadIdx.x], &sh);
        else
            bulk_cell<PREC, ODD>(a, L, idx, cg);
    }

    // warp-level aggregation of per-thread partial sums with equal keys, then
    // one block-table entry per key, then one global atomic per key and block
    __syncthreads();
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
        slot_add(&sh, a, key, v);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NSLOT; i += blockDim.x) {
        const uint32_t k2 = sh.key[i];
        if (k2 == SLOT_EMPTY) continue;
        double *g = global_acc(a, k2);
        const int nv = (k2 & KEY_WALL) ? 3 : 6;
        for (int k = 0; k < nv; ++k) atomicAdd(g + k, sh.v[i][k]);
    }
}

template <int PREC>
cudaError_t launch_prec(int parity, const SweepArgs &a, int grid, int block, cudaStream_t s) {
    const bool single = a.nlat == 1;
    if (parity) {
        if (single) sweep_kernel<PREC, 1, true><<<grid, block, 0, s>>>(a);
        else sweep_kernel<PREC, 1, false><<<grid, block, 0, s>>>(a);
    } else {
        if (single) sweep_kernel<PREC, 0, true><<<grid, block, 0, s>>>(a);
        else sweep_kernel<PREC, 0, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int PREC>
int max_blocks_prec(int parity, int block) {
    int nb = 0;
    if (parity)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<PREC, 1, false>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<PREC, 0, false>, block, 0);
    return nb;
}

}  // namespace

cudaError_t launch_sweep(int prec, int parity, const SweepArgs &a, int grid, int block,
                         cudaStream_t s) {
    switch (prec) {
    case LBM_F64: return launch_prec<LBM_F64>(parity, a, grid, block, s);
    case LBM_F32: return launch_prec<LBM_F32>(parity, a, grid, block, s);
    case LBM_F16_OFFSET: return launch_prec<LBM_F16_OFFSET>(parity, a, grid, block, s);
    case LBM_BF16_OFFSET: return launch_prec<LBM_BF16_OFFSET>(parity, a, grid, block, s);
    }
    return cudaErrorInvalidValue;
}

int sweep_max_active_blocks(int prec, int parity, int block) {
    switch (prec) {
    case LBM_F64: return max_blocks_prec<LBM_F64>(parity, block);
    case LBM_F32: return max_blocks_prec<LBM_F32>(parity, block);
    case LBM_F16_OFFSET: return max_blocks_prec<LBM_F16_OFFSET>(parity, block);
    case LBM_BF16_OFFSET: return max_blocks_prec<LBM_BF16_OFFSET>(parity, block);
    }
    return 0;
}

}  // namespace lbm
