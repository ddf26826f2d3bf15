// lbm_particles.cu -- everything of a time step besides the sweep:
//  * the rigid-body update of every particle (Sec. 4.3; the integrator is not
//    given in the paper: semi-implicit Euler on U and on the world-frame
//    angular momentum, quaternion exponential update, all FP64);
//  * the re-mapping of obstacle cells from the new poses (Sec. 4.2: a cell is
//    an obstacle cell iff its centre is inside a body), with equilibrium
//    refill of uncovered cells at rho0 and the surface velocity of the
//    previous time step (Sec. 4.2, last paragraph);
//  * field export in canonical form, population import, link compaction.
//
// Re-mapping runs over each body's box (union of its old and new bounding
// boxes, plus margin) in four passes separated by kernel boundaries:
//   A uncover: cells of body p no longer inside p become fluid (pid_prev = p);
//   B claim:   cells inside p take id min(id, p) (lowest index wins);
//   C fix-up:  every cell whose fluid/obstacle status changed is processed once
//              (by the body that uncovered or covered it) and its populations
//              are rewritten in the AA layout of the next sweep;
//   D flags:   flag bytes (obstacle / near-obstacle) are recomputed.
//
// AA layout between steps.  After an odd sweep the next sweep is even and
// reads f_q(x) from slot q of x, so a refill writes all 19 slots of x.  After
// an even sweep the next (odd) sweep reads f_p(z) from slot opp(p) of
// z - c_p if that cell is fluid, else from slot p of z.  Each lattice link
// {z, z' = z - c_p} therefore owns two slots A = (opp(p), z') and B = (p, z):
// with both cells fluid A holds f_p(z) and B holds f_opp(p)(z'); with only z
// fluid B holds f_p(z); with only z' fluid A holds f_opp(p)(z').  When a status
// changes, pass C reads the link's logical values under the old statuses and
// rewrites them under the new ones.  A free-slip wall cell (F_FSLIP) is not a
// bounce-back neighbour: the odd sweep pulls through its slots, which carry
// the values reflected at the wall (see the sweep); bodies keep off the fluid
// layer next to such walls, so pass C never meets one.
#include "lbm_internal.cuh"

namespace lbm {

namespace {

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ double min_image_rn(double d, int n, int periodic) {
    if (periodic) {
        const double h = 0.5 * (double)n;
        if (d > h)
            d = __dsub_rn(d, (double)n);
        else if (d < -h)
            d = __dadd_rn(d, (double)n);
    }
    return d;
}

// Cell centre (i,j,k) inside the body (Sec. 4.2), with p = R^T d and d the
// nearest-image displacement from the centre: ellipsoid
// (p0/a)^2 + (p1/b)^2 + (p2/c)^2 <= 1; spherocylinder of radius r = b and half
// length a along body x: t^2 + p1^2 + p2^2 <= r^2 with t = max(|p0| - (a - r), 0)
// (distance to the axis segment at most r).  Every operation rounds once, in
// the order written.
__device__ __forceinline__ bool inside_rn(const LatDev &L, const double *pos, const double R[9],
                                          const double *semi, int shape, int i, int j, int k) {
    const double d0 = min_image_rn(__dsub_rn((double)i, pos[0]), L.nx, L.px);
    const double d1 = min_image_rn(__dsub_rn((double)j, pos[1]), L.ny, L.py);
    const double d2 = min_image_rn(__dsub_rn((double)k, pos[2]), L.nz, L.pz);
    const double p0 = __dadd_rn(__dadd_rn(__dmul_rn(R[0], d0), __dmul_rn(R[3], d1)), __dmul_rn(R[6], d2));
    const double p1 = __dadd_rn(__dadd_rn(__dmul_rn(R[1], d0), __dmul_rn(R[4], d1)), __dmul_rn(R[7], d2));
    const double p2 = __dadd_rn(__dadd_rn(__dmul_rn(R[2], d0), __dmul_rn(R[5], d1)), __dmul_rn(R[8], d2));
    if (shape == 1) {
        const double r = semi[1];
        double t = __dsub_rn(fabs(p0), __dsub_rn(semi[0], r));
        if (t < 0.0) t = 0.0;
        const double s = __dadd_rn(__dadd_rn(__dmul_rn(t, t), __dmul_rn(p1, p1)), __dmul_rn(p2, p2));
        return s <= __dmul_rn(r, r);
    }
    const double t0 = __ddiv_rn(p0, semi[0]), t1 = __ddiv_rn(p1, semi[1]), t2 = __ddiv_rn(p2, semi[2]);
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(t0, t0), __dmul_rn(t1, t1)), __dmul_rn(t2, t2));
    return s <= 1.0;
}

// The same test decided in FP32 wherever that is safe: the FP32 value of s
// differs from the FP64 one by far less than 1e-4 for cells within a body's
// box (|d| below ~10^2, semi-axes >= ~1), so outside a band |s - 1| <= 1e-3
// the FP32 decision equals the FP64 one, and inside the band the exact FP64
// test decides.  The result is bit-identical to inside_rn.
// FP32 copy of a body's pose for that pre-test (from PartDev::bodyf:
// rotation, reciprocal semi-axes, centre, shape).  Both shapes share one
// form, s = max(|p0/a'| - h, 0)^2 + (p1/b)^2 + (p2/c)^2: h = 0 and a' = a for
// an ellipsoid, h = (a - r)/r and a' = b = c = r for a spherocylinder.
struct BodyF32 {
    float R[9];
    float inv[3];
    float pos[3], poslo[3];  // centre as a double-float
    float caph;
    int shape;
};

__device__ __forceinline__ void load_body_f32(const float *src, BodyF32 &b) {
    for (int k = 0; k < 9; ++k) b.R[k] = src[BF_R + k];
    for (int k = 0; k < 3; ++k) b.inv[k] = src[BF_INV + k];
    for (int k = 0; k < 3; ++k) b.pos[k] = src[BF_POS + k];
    for (int k = 0; k < 3; ++k) b.poslo[k] = src[BF_POSLO + k];
    b.caph = src[BF_CAPH];
    b.shape = (int)src[BF_SHAPE];
}

// Displacement x - x_C of a cell coordinate from a body centre held as the
// double-float (hi, lo): formed exactly enough (|error| ~ 2^-48 |x_C|), taken
// to the minimum image on a periodic axis, then rounded once to FP32.
// near_switch is set when |d| is within two cells of n/2, where the image
// choice is left to the FP64 test.
__device__ __forceinline__ float disp_f(int x, float hi, float lo, int n, int periodic, bool &near_switch) {
    df d = df_add_f(two_sum((float)x, -hi), -lo);
    if (periodic) {
        const float h = 0.5f * (float)n;
        near_switch = near_switch || fabsf(fabsf(d.hi) - h) < 2.0f;
        if (d.hi > h)
            d = df_add_f(d, -(float)n);
        else if (d.hi < -h)
            d = df_add_f(d, (float)n);
    }
    return d.hi;
}

// Exact inside test of the cell (i,j,k) for the body with double pose
// (pos, rotation R64), decided in FP32 where the FP32 value of s is far from
// 1; cells near the periodic image switch (|d| ~ n/2) always take the FP64
// test.
__device__ __forceinline__ bool inside_fast(const LatDev &L, const double *pos, const double *R64,
                                            const double *semi, const BodyF32 &b, int i, int j, int k) {
    // d rounded once from a double-float: |error(s)| < ~2e-4 for |d| < 100, semi-axes >= 1
    bool sw = false;
    const float d0 = disp_f(i, b.pos[0], b.poslo[0], L.nx, L.px, sw);
    const float d1 = disp_f(j, b.pos[1], b.poslo[1], L.ny, L.py, sw);
    const float d2 = disp_f(k, b.pos[2], b.poslo[2], L.nz, L.pz, sw);
    const float t0 = fmaxf(fabsf((b.R[0] * d0 + b.R[3] * d1 + b.R[6] * d2) * b.inv[0]) - b.caph, 0.0f);
    const float t1 = (b.R[1] * d0 + b.R[4] * d1 + b.R[7] * d2) * b.inv[1];
    const float t2 = (b.R[2] * d0 + b.R[5] * d1 + b.R[8] * d2) * b.inv[2];
    const float s = t0 * t0 + t1 * t1 + t2 * t2;
    if (!sw) {
        if (s < 0.999f) return true;
        if (s > 1.001f) return false;
    }
    return inside_rn(L, pos, R64, semi, b.shape, i, j, k);
}

// ---------------------------------------------------------------------------
// rigid-body update (one thread per body) and wall-force hand-over
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double sel3(int k, double v0, double v1, double v2) {
    return k == 0 ? v0 : (k == 1 ? v1 : v2);
}

// Entry e = 3i + j (row-major) of the rotation matrix of the unit quaternion
// (w, x, y, z) with v = (x, y, z), every product and sum rounded separately in
// a fixed order (the host builds the initial matrix in the same order, so the
// obstacle mapping is reproducible bit for bit): diagonal
// 1 - 2(v_a v_a + v_b v_b) over the two other axes a < b, off-diagonal
// 2(v_i v_j - eps_ijm w v_m).  Operands are selected, not branched on, so the
// nine lanes of a warp evaluate one instruction stream.
__device__ __forceinline__ double quat_entry_rn(int e, double w, double x, double y, double z) {
    const int i = e / 3, j = e - 3 * (e / 3);
    double pa, pb, pc, pd;
    if (i == j) {
        const int o1 = i == 0 ? 1 : 0, o2 = i == 2 ? 1 : 2;
        pa = pb = sel3(o1, x, y, z);
        pc = pd = sel3(o2, x, y, z);
    } else {
        const int m = 3 - i - j;
        const bool cyclic = j - i == 1 || j - i == -2;  // eps_ijm = +1
        pa = sel3(i, x, y, z);
        pb = sel3(j, x, y, z);
        pc = cyclic ? -w : w;
        pd = sel3(m, x, y, z);
    }
    const double X = __dadd_rn(__dmul_rn(pa, pb), __dmul_rn(pc, pd));
    const double t2 = __dmul_rn(2.0, X);
    return i == j ? __dsub_rn(1.0, t2) : t2;
}

// One warp per body (and per lattice for the wall loads): lane c reads and
// clears accumulator copy c and the warp sums the copies; then the body's
// update (Sec. 4.3) runs across the lanes -- lane k < 3 owns component k of
// every vector, lane e < 9 entry e of the rotation -- so that the FP64 work,
// which GB300 issues at a low rate per warp instruction, takes few
// instructions.  Every load is issued up front, every store at the end.
__device__ void rigid_unit(const RemapArgs &a, int warp, int lane) {
    static_assert(ACC_COPIES == 32, "one lane per accumulator copy");
    const unsigned full = 0xffffffffu;
    const PartDev &P = a.P;
    // warps [0, np) update the bodies, warps [np, np + nlat) hand over the walls
    if (warp >= P.np) {
        const int t = warp - P.np;
        if (t >= a.nlat) return;
        // the step counter (seed of the next sweep's stochastic rounding)
        if (t == 0 && lane == 0 && a.tick) *a.tick += 1u;
        double *w = a.wall_acc + 6 * ((size_t)t * ACC_COPIES + lane);
        double s[6];
        for (int k = 0; k < 6; ++k) s[k] = w[k];
        for (int k = 0; k < 6; ++k) w[k] = 0.0;
        for (int k = 0; k < 6; ++k) s[k] = warp_sum(s[k]);
        if (lane == 0) {
            for (int k = 0; k < 6; ++k) a.wall_last[6 * t + k] = s[k];
            // a non-finite population next to a wall shows in its momentum
            bool fin = true;
            for (int k = 0; k < 6; ++k) fin = fin && isfinite(s[k]);
            if (!fin) atomicOr(a.err, ERR_NONFINITE);
        }
        return;
    }
    const size_t t = (size_t)warp;
    if (lane == 0) P.changed[t] = 0;  // set again by this step's uncover / claim passes
    if (t == 0 && lane == 0 && a.chg_n) *a.chg_n = 0;  // the step's changed-cell list starts empty
    const int k = lane < 3 ? lane : 0;  // vector component of this lane (lanes >= 3 mirror 0, store nothing)
    const bool vec = lane < 3;
    // ---- loads
    const double pos = P.pos[3 * t + k], vel = P.vel[3 * t + k], om = P.om[3 * t + k], Lm = P.L[3 * t + k];
    const double Iinv = P.Iinv[3 * t + k], eF = P.extF[3 * t + k], eM = P.extM[3 * t + k];
    const double s0 = P.semi[3 * t], s1 = P.semi[3 * t + 1], s2 = P.semi[3 * t + 2];
    const double w = P.quat[4 * t], x = P.quat[4 * t + 1], y = P.quat[4 * t + 2], z = P.quat[4 * t + 3];
    const double *Rp = P.R64 + 9 * t;  // rotation of q, stored by the previous update
    const double Rr0 = Rp[3 * k], Rr1 = Rp[3 * k + 1], Rr2 = Rp[3 * k + 2];  // row k
    const double Rc0 = Rp[k], Rc1 = Rp[3 + k], Rc2 = Rp[6 + k];              // column k
    const double minv = P.minv[t];
    const int fixed = P.fixed[t];
    const LatDev &Lt = a.lat[P.cell[t]];
    const int dim = k == 0 ? Lt.nx : (k == 1 ? Lt.ny : Lt.nz);
    const int per = k == 0 ? Lt.px : (k == 1 ? Lt.py : Lt.pz);
    double hs[6];  // F_h, M_h: the sweep's copies, summed
    {
        double *acc = P.acc + 6 * (t * ACC_COPIES + lane);
        for (int c = 0; c < 6; ++c) hs[c] = acc[c];
        for (int c = 0; c < 6; ++c) acc[c] = 0.0;
        for (int c = 0; c < 6; ++c) hs[c] = warp_sum(hs[c]);
    }
    const double hF = sel3(k, hs[0], hs[1], hs[2]), hM = sel3(k, hs[3], hs[4], hs[5]);
    if (vec) {
        P.last[6 * t + k] = hF;
        P.last[6 * t + 3 + k] = hM;
        P.pos_old[3 * t + k] = pos;
        P.vel_old[3 * t + k] = vel;
        P.om_old[3 * t + k] = om;
    }
    if (lane < 4) P.quat_old[4 * t + lane] = lane == 0 ? w : sel3(lane - 1, x, y, z);
    const double F = hF + eF, M = hM + eM;
    bool finite = isfinite(F) && isfinite(M);
    // old box half extent along k (FP32; the box only has to contain the
    // body): ellipsoid sqrt(sum_j (R_kj s_j)^2); spherocylinder (radius
    // s1, half length s0) |R_k0| (s0 - s1) + s1, the same form with the
    // ellipsoid's first semi-axis replaced by s1 and the segment term added
    const bool capsule = P.bodyf[BF_STRIDE * t + BF_SHAPE] != 0.0f;
    const float sf0 = capsule ? (float)s1 : (float)s0, sf1 = (float)s1, sf2 = (float)s2;
    const float seg = capsule ? (float)(s0 - s1) : 0.0f;
    auto half = [&](float r0, float r1, float r2) {
        const float e0 = r0 * sf0, e1 = r1 * sf1, e2 = r2 * sf2;
        return (sqrtf(e0 * e0 + e1 * e1 + e2 * e2) + fabsf(r0) * seg) * 1.0001f;
    };
    const float hold = half((float)Rr0, (float)Rr1, (float)Rr2);
    double posn = pos, veln = vel, omn = om, Ln = Lm, wn = w, xn = x, yn = y, zn = z;
    if (!fixed) {
        // divisions are replaced by the host's reciprocals of mass and inertia
        veln = vel + F * minv;
        posn = pos + veln;
        Ln = Lm + M;
        // omega = R diag(1/I) R^T L with the orientation before the update
        const double L0 = __shfl_sync(full, Ln, 0), L1 = __shfl_sync(full, Ln, 1), L2 = __shfl_sync(full, Ln, 2);
        const double lb = (Rc0 * L0 + Rc1 * L1 + Rc2 * L2) * Iinv;
        const double b0 = __shfl_sync(full, lb, 0), b1 = __shfl_sync(full, lb, 1), b2 = __shfl_sync(full, lb, 2);
        omn = Rr0 * b0 + Rr1 * b1 + Rr2 * b2;
        const double o0 = __shfl_sync(full, omn, 0), o1 = __shfl_sync(full, omn, 1), o2 = __shfl_sync(full, omn, 2);
        const double th2 = o0 * o0 + o1 * o1 + o2 * o2;
        // exp(Omega/2) = (cos(th/2), sin(th/2) Omega/th); for the small angles of
        // one lattice step the Maclaurin series of cos x and sin x / x in
        // x^2 = th^2/4, truncated after x^8 (remainder < 1e-19 for th < 0.02)
        double ch, shr;  // cos(th/2), sin(th/2)/th
        if (th2 < 4e-4) {
            const double x2 = 0.25 * th2;
            ch = 1.0 + x2 * (-1.0 / 2 + x2 * (1.0 / 24 + x2 * (-1.0 / 720 + x2 * (1.0 / 40320))));
            shr = 0.5 * (1.0 + x2 * (-1.0 / 6 + x2 * (1.0 / 120 + x2 * (-1.0 / 5040 + x2 * (1.0 / 362880)))));
        } else {
            const double th = sqrt(th2);
            double sh;
            sincos(0.5 * th, &sh, &ch);
            shr = sh / th;
        }
        const double d0 = ch, d1 = o0 * shr, d2 = o1 * shr, d3 = o2 * shr;
        const double n0 = d0 * w - (d1 * x + d2 * y + d3 * z);
        const double n1 = d0 * x + w * d1 + (d2 * z - d3 * y);
        const double n2 = d0 * y + w * d2 + (d3 * x - d1 * z);
        const double n3 = d0 * z + w * d3 + (d1 * y - d2 * x);
        // renormalise: a product of unit quaternions has |n|^2 = 1 + d with d
        // at rounding level, and one Newton step for 1/sqrt from 1 gives
        // 1.5 - 0.5 |n|^2, exact to O(d^2)
        const double nn = n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3;
        const double rn = fabs(nn - 1.0) < 1e-6 ? 1.5 - 0.5 * nn : 1.0 / sqrt(nn);
        wn = n0 * rn;
        xn = n1 * rn;
        yn = n2 * rn;
        zn = n3 * rn;
        if (per) {
            if (posn >= dim)
                posn -= dim;
            else if (posn < 0.0)
                posn += dim;
        }
        finite = finite && isfinite(posn) && isfinite(omn);
    }
    if (!__all_sync(full, finite) && lane == 0) atomicOr(a.err, ERR_NONFINITE);
    // rotation of the new orientation (lane e < 9: entry e), rounded as the
    // mapping's exact inside test expects, and its FP32 copy
    const double Re = quat_entry_rn(lane < 9 ? lane : 0, wn, xn, yn, zn);
    const float Rf = (float)Re;
    float *bf = P.bodyf + BF_STRIDE * t;
    if (lane < 9) {
        P.R64[9 * t + lane] = Re;
        bf[BF_R + lane] = Rf;
    }
    const float hnew = half(__shfl_sync(full, Rf, 3 * k), __shfl_sync(full, Rf, 3 * k + 1),
                            __shfl_sync(full, Rf, 3 * k + 2));
    if (!fixed) {
        if (vec) {
            P.pos[3 * t + k] = posn;
            P.vel[3 * t + k] = veln;
            P.om[3 * t + k] = omn;
            P.L[3 * t + k] = Ln;
        }
        if (lane < 4) P.quat[4 * t + lane] = lane == 0 ? wn : sel3(lane - 1, xn, yn, zn);
    }
    if (!vec) return;
    // FP32 copies of the new centre (double-float), velocity and angular
    // velocity for the re-mapping pre-test and the sweep's bounce-back
    const df c = df_from_double(posn);
    bf[BF_POS + k] = c.hi;
    bf[BF_POSLO + k] = c.lo;
    bf[BF_U + k] = (float)veln;
    bf[BF_W + k] = (float)omn;
    // re-mapping box along k: union of the old and new bounding boxes plus a
    // margin of two cells, in FP32 with a slack far above its rounding
    const float posf = c.hi, coldf = (float)pos;
    // a body must keep off the fluid layer next to a free-slip wall
    const int fsk = k == 0 ? Lt.fsx : (k == 1 ? Lt.fsy : Lt.fsz);
    if (fsk && (posf - hnew < 1.5f || posf + hnew > (float)dim - 2.5f)) atomicOr(a.err, ERR_FSLIP_BODY);
    float lo = fminf(coldf - hold, posf - hnew) - 1e-3f;
    float hi = fmaxf(coldf + hold, posf + hnew) + 1e-3f;
    // a wrapped centre makes the two boxes an image apart: use the new one
    if (per && fabsf(coldf - posf) > 0.5f * (float)dim) {
        lo = fminf(posf - hnew, posf - hold) - 1e-3f;
        hi = fmaxf(posf + hnew, posf + hold) + 1e-3f;
    }
    int ilo = (int)floorf(lo) - 2, ihi = (int)ceilf(hi) + 2;
    if (!isfinite(lo) || !isfinite(hi)) { ilo = 0; ihi = -1; }
    if (per) {
        if (ihi - ilo + 1 > dim) { ilo = 0; ihi = dim - 1; }
    } else {
        ilo = max(ilo, 0);
        ihi = min(ihi, dim - 1);
    }
    P.region[6 * t + k] = ilo;
    P.region[6 * t + 3 + k] = max(ihi - ilo + 1, 0);
    // the cylinder the re-mapping passes visit this step (BF_TUBE_H/R): the
    // largest displacement of a body point in the step is at most
    // |U| + |Omega| * (largest semi-axis) (a fixed body keeps its pose)
    {
        const float du = fixed ? 0.0f : (float)veln, wk = fixed ? 0.0f : (float)omn;
        const float d0 = __shfl_sync(0x7u, du, 0), d1 = __shfl_sync(0x7u, du, 1), d2 = __shfl_sync(0x7u, du, 2);
        const float w0 = __shfl_sync(0x7u, wk, 0), w1 = __shfl_sync(0x7u, wk, 1), w2 = __shfl_sync(0x7u, wk, 2);
        if (lane == 0) {
            const float smax = fmaxf((float)s0, fmaxf((float)s1, (float)s2));
            float delta = sqrtf(d0 * d0 + d1 * d1 + d2 * d2) + sqrtf(w0 * w0 + w1 * w1 + w2 * w2) * smax;
            if (!(delta < 1e6f)) delta = 1e6f;  // non-finite state: every row whole (the step is reported)
            bf[BF_TUBE_H] = (float)s0 + 2.0f + delta;
            bf[BF_TUBE_R] = fmaxf((float)s1, (float)s2) + 2.0f + delta;
        }
    }
}

__global__ void rigid_body_kernel(RemapArgs a) {
    pdl_enter();
    rigid_unit(a, (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// re-mapping passes
// ---------------------------------------------------------------------------

struct RegionCell {
    int i, j, k;
    int idx;  // index within the lattice
};

__device__ __forceinline__ int modc(int v, int n) {
    const int m = v % n;
    return m < 0 ? m + n : m;
}

// v mod n for v in [-n, 2n) without a division (a box origin lies within one
// period of its body's wrapped centre and a box spans at most one period),
// with the division kept for any other v.
__device__ __forceinline__ int wrap_box(int v, int n) {
    if (v >= 0 && v < n) return v;
    if (v < 0 && v >= -n) return v + n;
    if (v >= n && v < 2 * n) return v - n;
    return modc(v, n);
}

// Cell of a box from its box coordinates (r0 along x, row r1 + e1 r2).
__device__ __forceinline__ void box_cell(const int *reg, const LatDev &L, int r0, int r1, int r2, RegionCell &c) {
    c.i = wrap_box(reg[0] + r0, L.nx);
    c.j = wrap_box(reg[1] + r1, L.ny);
    c.k = wrap_box(reg[2] + r2, L.nz);
    c.idx = c.i + L.nx * (c.j + L.ny * c.k);
}

// Cells of a re-mapping box that the passes visit: the box's rows (y, z) and
// in each row the x interval that meets the body's cylinder (BF_TUBE_H/R
// about the body x axis through the centre, in the frame of the box, whose
// origin reg[0..2] is unwrapped around the centre).  The cylinder holds the
// body (an ellipsoid (a, b, c) lies within radius max(b, c) of its x axis and
// |x| <= a; a spherocylinder (L/2, r, r) within radius r and |x| <= L/2),
// widened by the step's largest displacement of a body point and two cells:
// every cell a pass can change (uncovered, claimed, refilled, re-flagged) is
// inside, so the passes give the same maps as over the whole box.  The
// interval is computed in FP32 and widened by one more cell on each side.
// Returns x0 > x1 for a row that misses the cylinder.
__device__ __forceinline__ void row_interval(const int *reg, const float *bf, int r1, int r2, int &x0, int &x1) {
    const float H = bf[BF_TUBE_H], rho = bf[BF_TUBE_R];
    const float tx = bf[BF_R + 0], ty = bf[BF_R + 3], tz = bf[BF_R + 6];
    const float cx = bf[BF_POS] - (float)reg[0];
    const float dy = (float)(reg[1] + r1) - bf[BF_POS + 1];
    const float dz = (float)(reg[2] + r2) - bf[BF_POS + 2];
    const float s0 = ty * dy + tz * dz;  // axial coordinate at X = x - x_C = 0
    float lo = -3.0e38f, hi = 3.0e38f;
    x0 = 0;
    x1 = -1;
    // axial: |tx X + s0| <= H
    if (fabsf(tx) > 1e-6f) {
        const float ea = (-H - s0) / tx, eb = (H - s0) / tx;
        lo = fminf(ea, eb);
        hi = fmaxf(ea, eb);
    } else if (fabsf(s0) > H) {
        return;
    }
    // radial: |d|^2 - (t.d)^2 <= rho^2, a quadratic (1 - tx^2) X^2 - 2 tx s0 X + C <= 0
    const float A = 1.0f - tx * tx, B = -2.0f * tx * s0, C = dy * dy + dz * dz - s0 * s0 - rho * rho;
    if (A > 1e-6f) {
        const float disc = B * B - 4.0f * A * C;
        if (disc < 0.0f) return;
        const float sq = sqrtf(disc);
        lo = fmaxf(lo, (-B - sq) / (2.0f * A));
        hi = fminf(hi, (-B + sq) / (2.0f * A));
    } else if (C > 0.0f) {
        return;
    }
    if (!(lo <= hi)) return;
    x0 = max(0, (int)fmaxf(floorf(cx + lo) - 1.0f, -1.0f));
    x1 = min(reg[3] - 1, (int)fminf(ceilf(cx + hi) + 1.0f, (float)reg[3]));
}

// Threads per block of the re-mapping passes.
constexpr int REMAP_BLOCK = 256;

// The region passes work on np * bpb units of one block each: unit u covers
// body p = u / bpb.  The separate kernels run one unit per block; the fused
// kernel loops its blocks over the units.
struct RegionLoop {
    int p, first, stride;
};

__device__ __forceinline__ RegionLoop region_loop(int unit, int bpb) {
    RegionLoop l;
    l.p = unit / bpb;
    l.first = (unit % bpb) * blockDim.x + threadIdx.x;
    l.stride = bpb * blockDim.x;
    return l;
}

// The cells of a box that lie in its rows' cylinder intervals, each handed
// once to f(r0, r1, r2) (box coordinates: r0 along x, row r1 + e1 r2, e1 the
// box's extent in y).  The warps of a body's units take the box's rows in
// batches of up to 32 (fewer when the box has fewer than 32 rows per warp,
// so that every warp gets rows): each lane of a batch finds the interval of
// one row, a warp prefix sum lays the rows' cells end to end, and
// the lanes take that list 32 cells at a time (a lane finds the row of its
// cell by binary search over the prefix sums), so a short row does not leave
// most of a warp idle and a row missing the cylinder costs one lane's
// interval test.  Called by whole warps; f runs on the lanes that hold a
// cell.  f returns a cell (index in the flag arena) to append to the step's
// changed-cell list, or -1; the warp appends its cells with one atomic.
template <class F>
__device__ __forceinline__ void for_tube_cells(const RemapArgs &a, const int *reg, const float *bfp,
                                               const RegionLoop &rl, F &&f) {
    constexpr unsigned FULL = 0xffffffffu;
    const int rows = reg[4] * reg[5];
    const int lane = threadIdx.x & 31;
    const int nw = rl.stride >> 5;
    const int batch = min(32, max(1, (rows + nw - 1) / nw));
    for (int rb = (rl.first >> 5) * batch; rb < rows; rb += nw * batch) {
        const int r = rb + lane;
        const int r1 = r % reg[4], r2 = r / reg[4];
        int x0 = 0, x1 = -1;
        if (lane < batch && r < rows) row_interval(reg, bfp, r1, r2, x0, x1);
        const int len = x1 >= x0 ? x1 - x0 + 1 : 0;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        for (int jb = 0; jb < total; jb += 32) {
            const int j = jb + lane;
            // row of cell j: the first lane whose inclusive sum exceeds j
            int l = 0;
#pragma unroll
            for (int b = 16; b; b >>= 1) {
                const int v = __shfl_sync(FULL, incl, l + b - 1);
                if (v <= j) l += b;
            }
            l = l < 31 ? l : 31;
            const int rx0 = __shfl_sync(FULL, x0, l);
            const int rstart = __shfl_sync(FULL, incl - len, l);
            const int c1 = __shfl_sync(FULL, r1, l), c2 = __shfl_sync(FULL, r2, l);
            long long add = -1;
            if (j < total) add = f(rx0 + (j - rstart), c1, c2);
            const unsigned bal = __ballot_sync(FULL, add >= 0);
            if (bal && a.chg) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(a.chg_n, (uint32_t)__popc(bal));
                base = __shfl_sync(FULL, base, 0) + (uint32_t)__popc(bal & ((1u << lane) - 1u));
                if (add >= 0 && (long long)base < a.chg_cap) a.chg[base] = (uint32_t)add;
            }
        }
    }
}

// Sets F_CHANGED on cell cg (flag byte) and tells whether this call set it:
// an atomic OR on the byte's 32-bit word (the passes touch flag bytes only
// through this), so a cell changed by several bodies is listed once.
__device__ __forceinline__ bool mark_changed(uint8_t *flags, long long cg) {
    uint32_t *word = reinterpret_cast<uint32_t *>(flags + (cg & ~3ll));
    const uint32_t bit = (uint32_t)F_CHANGED << (8 * (int)(cg & 3));
    return !(atomicOr(word, bit) & bit);
}

template <int PASS>
__device__ void remap_region(const RemapArgs &a, int unit, int bpb) {
    const RegionLoop rl = region_loop(unit, bpb);
    const int p = rl.p;
    const PartDev &P = a.P;
    if (p >= P.np) return;
    const int *reg = P.region + 6 * p;
    const int vol = reg[3] * reg[4] * reg[5];
    if (vol <= 0) return;
    const LatDev &L = a.lat[P.cell[p]];
    const double *pos = P.pos + 3 * p, *semi = P.semi + 3 * p, *R64 = P.R64 + 9 * (size_t)p;
    BodyF32 bf;
    const float *bfp = P.bodyf + BF_STRIDE * (size_t)p;
    load_body_f32(bfp, bf);
    for_tube_cells(a, reg, bfp, rl, [&](int r0, int r1, int r2) -> long long {
        RegionCell c;
        box_cell(reg, L, r0, r1, r2, c);
        const long long cg = L.c_off + c.idx;
        if (PASS == 2) {  // a single body: uncover and claim in one pass
            const uint32_t cur = a.pid[cg];
            if (cur == (uint32_t)p) {
                if (!inside_fast(L, pos, R64, semi, bf, c.i, c.j, c.k)) {
                    a.pid[cg] = PID_FLUID;
                    a.pid_prev[cg] = (uint32_t)p;
                    P.changed[p] = 1;
                    return mark_changed(a.flags, cg) ? cg : -1;
                }
            } else if (cur == PID_FLUID && inside_fast(L, pos, R64, semi, bf, c.i, c.j, c.k)) {
                a.pid[cg] = (uint32_t)p;
                P.changed[p] = 1;
                return mark_changed(a.flags, cg) ? cg : -1;
            }
        } else if (PASS == 0) {  // uncover
            if (a.pid[cg] == (uint32_t)p && !inside_fast(L, pos, R64, semi, bf, c.i, c.j, c.k)) {
                a.pid[cg] = PID_FLUID;
                a.pid_prev[cg] = (uint32_t)p;
                P.changed[p] = 1;
                return mark_changed(a.flags, cg) ? cg : -1;
            }
        } else {  // claim
            // a cell of this body (still inside: the uncover pass ran) or of
            // a lower-index body (which keeps it) needs no test, nor a wall cell
            const uint32_t cur = a.pid[cg];
            if (cur <= (uint32_t)p || (cur >= PID_WALL && cur != PID_FLUID)) return -1;
            if (inside_fast(L, pos, R64, semi, bf, c.i, c.j, c.k)) {
                const uint32_t old = atomicMin(&a.pid[cg], (uint32_t)p);
                // a new obstacle cell, or one taken from a higher-index body
                // (the neighbours' first-body links change)
                if (old > (uint32_t)p) {
                    P.changed[p] = 1;
                    return mark_changed(a.flags, cg) ? cg : -1;
                }
            }
        }
        return -1;
    });
}

template <int PASS>
__global__ void __launch_bounds__(REMAP_BLOCK, 4) remap_region_kernel(RemapArgs a, int bpb) {
    pdl_enter();
    remap_region<PASS>(a, blockIdx.x, bpb);
}

// Equilibrium offset f^eq_q(rho0, u) - w_q rho0 (Eq. fequ_Incompr).
__device__ __forceinline__ double geq(int q, double rho0, const double u[3]) {
    const double cu = cx(q) * u[0] + cy(q) * u[1] + cz(q) * u[2];
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return wq(q) * rho0 * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

// Refill velocity of an uncovered cell: surface velocity of its previous
// owner, from that body's state before this step's update (zero at rest).
__device__ __forceinline__ void refill_velocity(const RemapArgs &a, const LatDev &L, uint32_t owner,
                                                bool at_rest, int i, int j, int k, double u[3]) {
    u[0] = u[1] = u[2] = 0.0;
    if (at_rest || owner >= (uint32_t)a.P.np) return;
    const double *pos = a.P.pos_old + 3 * owner, *U = a.P.vel_old + 3 * owner,
                 *W = a.P.om_old + 3 * owner;
    double r[3];
    r[0] = (double)i - pos[0];
    r[1] = (double)j - pos[1];
    r[2] = (double)k - pos[2];
    const int dims[3] = {L.nx, L.ny, L.nz}, per[3] = {L.px, L.py, L.pz};
    for (int m = 0; m < 3; ++m)
        if (per[m]) {
            if (r[m] > 0.5 * dims[m]) r[m] -= dims[m];
            else if (r[m] < -0.5 * dims[m]) r[m] += dims[m];
        }
    u[0] = U[0] + (W[1] * r[2] - W[2] * r[1]);
    u[1] = U[1] + (W[2] * r[0] - W[0] * r[2]);
    u[2] = U[2] + (W[0] * r[1] - W[1] * r[0]);
}

struct Coord {
    int i, j, k;
};

__device__ __forceinline__ int lin(const LatDev &L, int i, int j, int k) {
    return wrapc(i, L.nx) + L.nx * (wrapc(j, L.ny) + L.ny * wrapc(k, L.nz));
}

// Pass C for one status-changed cell x (see the file comment).
template <int PREC, int NEXT_ODD>
__device__ void fixup_cell(const RemapArgs &a, const LatDev &L, int i, int j, int k, bool at_rest) {
    using S = Store<PREC>;
    using T = typename S::T;
    T *base = reinterpret_cast<T *>(a.f) + L.f_off;
    const long long np = L.npad;
    const int x = i + L.nx * (j + L.ny * k);
    const long long cx0 = L.c_off;
    const bool old_f = !(a.flags[cx0 + x] & F_SOLID);
    const bool new_f = a.pid[cx0 + x] == PID_FLUID;
    if (old_f == new_f) return;
    double ux[3];
    if (new_f) refill_velocity(a, L, a.pid_prev[cx0 + x], at_rest, i, j, k, ux);

    if (!NEXT_ODD) {
        if (new_f)
#pragma unroll
            for (int q = 0; q < Q; ++q) S::st(base + q * np + x, (typename S::C)geq(q, L.rho0, ux));
        return;
    }
    if (new_f) S::st(base + x, (typename S::C)geq(0, L.rho0, ux));
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int zi = i - cx(q), zj = j - cy(q), zk = k - cz(q);
        const int z = lin(L, zi, zj, zk);
        const bool old_z = !(a.flags[cx0 + z] & F_SOLID);
        const bool new_z = a.pid[cx0 + z] == PID_FLUID;
        if (old_z != new_z && z < x) continue;  // the lower index handles a doubly changed link
        T *A = base + opp(q) * np + z;
        T *B = base + q * np + x;
        const double va = (double)S::ld(A), vb = (double)S::ld(B);
        double v1 = 0.0, v2 = 0.0;
        if (new_f) v1 = old_f ? (old_z ? va : vb) : geq(q, L.rho0, ux);
        if (new_z) {
            if (old_z) {
                v2 = old_f ? vb : va;
            } else {
                double uz[3];
                refill_velocity(a, L, a.pid_prev[cx0 + z], at_rest, wrapc(zi, L.nx), wrapc(zj, L.ny),
                                wrapc(zk, L.nz), uz);
                v2 = geq(opp(q), L.rho0, uz);
            }
        }
        if (new_f && new_z) {
            S::st(A, (typename S::C)v1);
            S::st(B, (typename S::C)v2);
        } else if (new_f) {
            S::st(B, (typename S::C)v1);
        } else if (new_z) {
            S::st(A, (typename S::C)v2);
        }
    }
}

template <int PREC, int NEXT_ODD>
__device__ void fixup_region(const RemapArgs &a, int unit, int bpb) {
    const RegionLoop rl = region_loop(unit, bpb);
    const int p = rl.p;
    const PartDev &P = a.P;
    if (p >= P.np) return;
    // every changed cell and its neighbours lie in the box of the body that
    // changed it: a body that changed nothing has nothing to fix up here
    if (!P.changed[p]) return;
    const int *reg = P.region + 6 * p;
    const float *bfp = P.bodyf + BF_STRIDE * (size_t)p;
    const LatDev &L = a.lat[P.cell[p]];
    for_tube_cells(a, reg, bfp, rl, [&](int r0, int r1, int r2) -> long long {
        RegionCell c;
        box_cell(reg, L, r0, r1, r2, c);
        const long long cg = L.c_off + c.idx;
        if (!(a.flags[cg] & F_CHANGED)) return -1;
        const bool old_f = !(a.flags[cg] & F_SOLID);
        const uint32_t id = a.pid[cg];
        const bool new_f = id == PID_FLUID;
        if (old_f == new_f) return -1;
        // exactly one body handles each changed cell: its uncoverer or its new owner
        const uint32_t owner = new_f ? a.pid_prev[cg] : id;
        if (owner != (uint32_t)p) return -1;
        fixup_cell<PREC, NEXT_ODD>(a, L, c.i, c.j, c.k, false);
        return -1;
    });
}

// Wall cell (i,j,k) all of whose wall layers are free-slip walls.
__device__ __forceinline__ bool free_slip_cell(const LatDev &L, int i, int j, int k) {
    const bool lx = !L.px && (i == 0 || i == L.nx - 1);
    const bool ly = !L.py && (j == 0 || j == L.ny - 1);
    const bool lz = !L.pz && (k == 0 || k == L.nz - 1);
    return (lx || ly || lz) && (!lx || L.fsx) && (!ly || L.fsy) && (!lz || L.fsz);
}

// Flag byte of cell (i,j,k) from the particle-id map, and for a fluid cell
// its link word (LK_* layout) and the first body among its neighbours.  A
// link into a free-slip wall cell sets the wall bit only (not the solid bit):
// it reflects, and the odd step pulls through it.
__device__ __forceinline__ uint8_t flag_of(const LatDev &L, const uint32_t *pid, long long coff, int i,
                                           int j, int k, uint64_t &links, uint32_t &p0) {
    links = 0;
    p0 = PID_FLUID;
    const uint32_t id = pid[coff + i + L.nx * (j + L.ny * k)];
    if (id != PID_FLUID)
        return id >= PID_WALL ? (F_SOLID | F_WALL | (free_slip_cell(L, i, j, k) ? F_FSLIP : 0)) : F_SOLID;
    bool near = false, only_lo = true, only_hi = true;
    uint32_t solid = 0, wall = 0, body = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const int n = lin(L, i + cx(q), j + cy(q), k + cz(q));
        const uint32_t nid = pid[coff + n];
        if (nid >= PID_WALL && nid != PID_FLUID &&
            free_slip_cell(L, wrapc(i + cx(q), L.nx), wrapc(j + cy(q), L.ny), wrapc(k + cz(q), L.nz))) {
            wall |= 1u << q;
            near = true;
            only_lo = only_hi = false;
            continue;
        }
        if (nid != PID_FLUID) {
            solid |= 1u << q;
            if (nid >= PID_WALL) {
                wall |= 1u << q;
            } else {
                if (p0 == PID_FLUID) p0 = nid;
                if (nid == p0) body |= 1u << q;
            }
            near = true;
            // a wall cell hit along c_q must be in the layer c_q points to
            only_lo = only_lo && nid == PID_WALL_YLO && cy(q) < 0;
            only_hi = only_hi && nid == PID_WALL_YHI && cy(q) > 0;
        } else {
            // every direction into the layer must hit it: the layer is a full plane
            only_lo = only_lo && !(cy(q) < 0 && j == 1 && !L.py);
            only_hi = only_hi && !(cy(q) > 0 && j == L.ny - 2 && !L.py);
        }
    }
    if (!near) return 0;
    links = (uint64_t)solid | ((uint64_t)wall << LK_WALL) | ((uint64_t)body << LK_BODY);
    if (only_lo && j == 1 && !L.py) return F_NEAR | F_YLO;
    if (only_hi && j == L.ny - 2 && !L.py) return F_NEAR | F_YHI;
    return F_NEAR;
}

__device__ void flags_region(const RemapArgs &a, int unit, int bpb) {
    const RegionLoop rl = region_loop(unit, bpb);
    const int p = rl.p;
    const PartDev &P = a.P;
    if (p >= P.np) return;
    if (!P.changed[p]) return;  // no owner changed in this box: flags and links stand
    const int *reg = P.region + 6 * p;
    const float *bfp = P.bodyf + BF_STRIDE * (size_t)p;
    const LatDev &L = a.lat[P.cell[p]];
    for_tube_cells(a, reg, bfp, rl, [&](int r0, int r1, int r2) -> long long {
        RegionCell c;
        box_cell(reg, L, r0, r1, r2, c);
        const long long cg = L.c_off + c.idx;
        if (a.flags[cg] & F_WALL) return -1;
        uint64_t lk;
        uint32_t p0;
        const uint8_t f = flag_of(L, a.pid, L.c_off, c.i, c.j, c.k, lk, p0);
        a.flags[cg] = f;
        a.links[cg] = lk;
        a.nbody[cg] = p0;
        // a cell turning non-bulk marks its tile; marks are cleared only by a
        // recount (launch_tile_bits), so a stale mark costs the flagged path,
        // never a missed cell
        if (f && a.tbits) {
            const int t = L.tile0 + c.idx / a.tile;
            atomicOr(a.tbits + (t >> 5), 1u << (t & 31));
        }
        return -1;
    });
}

// The fix-up and flags passes over the step's changed-cell list (the
// separate launches; the fused kernel keeps the passes over the boxes): every
// cell whose owner changed is listed once, and only it and its neighbours can
// need new populations, flags or link words.
struct ListedCell {
    const LatDev *L;
    int i, j, k, idx;
};

__device__ __forceinline__ ListedCell listed_cell(const RemapArgs &a, uint32_t cell) {
    int li = 0;
    if (a.nlat > 1) {
        int lo = 0, hi = a.nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.lat[mid].c_off <= (long long)cell) lo = mid; else hi = mid - 1;
        }
        li = lo;
    }
    ListedCell c;
    c.L = a.lat + li;
    c.idx = (int)((long long)cell - c.L->c_off);
    const uint32_t yz = c.L->divx.div((uint32_t)c.idx);
    c.i = c.idx - (int)yz * c.L->nx;
    c.k = (int)c.L->divxy.div((uint32_t)c.idx);
    c.j = (int)yz - c.k * c.L->ny;
    return c;
}

__device__ __forceinline__ uint32_t changed_count(const RemapArgs &a) {
    const uint32_t n = *a.chg_n;
    return (long long)n < a.chg_cap ? n : (uint32_t)a.chg_cap;
}

// Pass C over the list: one thread per changed cell.
template <int PREC, int NEXT_ODD>
__global__ void fixup_list_kernel(RemapArgs a) {
    pdl_enter();
    const uint32_t n = changed_count(a);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const uint32_t cell = a.chg[t];
        const bool old_f = !(a.flags[cell] & F_SOLID);
        const bool new_f = a.pid[cell] == PID_FLUID;
        if (old_f == new_f) continue;  // owner changed between bodies: populations stay dropped
        const ListedCell c = listed_cell(a, cell);
        fixup_cell<PREC, NEXT_ODD>(a, *c.L, c.i, c.j, c.k, false);
    }
}

// Pass D over the list: one thread per (changed cell, direction q), for the
// cell x + c_q (q = 0: the cell itself); a cell next to several changed cells
// is recomputed by several threads, which write the same values.  Neighbours
// outside a non-periodic lattice face are skipped (wall layers keep their
// flags).
__global__ void flags_list_kernel(RemapArgs a) {
    pdl_enter();
    const uint32_t n = changed_count(a);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n * Q; t += gridDim.x * blockDim.x) {
        const uint32_t cell = a.chg[t / Q];
        const int q = (int)(t % Q);
        const ListedCell c = listed_cell(a, cell);
        const LatDev &L = *c.L;
        const int i = c.i + cx(q), j = c.j + cy(q), k = c.k + cz(q);
        if ((!L.px && (i < 0 || i >= L.nx)) || (!L.py && (j < 0 || j >= L.ny)) || (!L.pz && (k < 0 || k >= L.nz)))
            continue;
        const int wi = wrapc(i, L.nx), wj = wrapc(j, L.ny), wk = wrapc(k, L.nz);
        const int idx = wi + L.nx * (wj + L.ny * wk);
        const long long cg = L.c_off + idx;
        if (a.flags[cg] & F_WALL) continue;
        uint64_t lk;
        uint32_t p0;
        const uint8_t f = flag_of(L, a.pid, L.c_off, wi, wj, wk, lk, p0);
        a.flags[cg] = f;
        a.links[cg] = lk;
        a.nbody[cg] = p0;
        if (f && a.tbits) {
            const int tt = L.tile0 + idx / a.tile;
            atomicOr(a.tbits + (tt >> 5), 1u << (tt & 31));
        }
    }
}

// Grid-wide barrier of the fused re-mapping kernel, whose blocks are all
// resident (cooperative launch).  count: blocks arrived at the current
// barrier; gen: barriers completed.  Thread 0 of each block reads gen before
// it arrives (gen cannot move before every block has arrived); the last block
// to arrive resets count and advances gen, the others poll gen, at most
// b->limit times (2^20 when 0).  Returns false after setting ERR_TIMEOUT when
// the poll ran out.
__device__ bool grid_barrier(GridBar *b, uint32_t *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        const unsigned g = *(volatile unsigned *)&b->gen;
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned lim = b->limit ? b->limit : (1u << 20);
            unsigned it = 0;
            while (*(volatile unsigned *)&b->gen == g) {
                if (++it >= lim) {
                    good = 0;
                    atomicOr(err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}


// The whole re-mapping step in one cooperative launch: rigid-body update of
// every body (and wall hand-over), then uncover, claim, population fix-up and
// flags, each pass over all np * bpb region units, with a grid barrier between
// passes in place of the kernel boundaries of the separate launches.  The
// arithmetic of every pass is that of the separate kernels.
template <int PREC, int NEXT_ODD>
__global__ void __launch_bounds__(REMAP_BLOCK) remap_fused_kernel(RemapArgs a, int bpb, GridBar *bar) {
    pdl_enter();
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int lane = threadIdx.x & 31;
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < a.P.np + a.nlat; w += nwarps)
        rigid_unit(a, w, lane);
    const int units = bpb * a.P.np;
    if (!grid_barrier(bar, a.err)) return;
    for (int u = blockIdx.x; u < units; u += gridDim.x) remap_region<0>(a, u, bpb);
    if (!grid_barrier(bar, a.err)) return;
    for (int u = blockIdx.x; u < units; u += gridDim.x) remap_region<1>(a, u, bpb);
    if (!grid_barrier(bar, a.err)) return;
    for (int u = blockIdx.x; u < units; u += gridDim.x) fixup_region<PREC, NEXT_ODD>(a, u, bpb);
    if (!grid_barrier(bar, a.err)) return;
    for (int u = blockIdx.x; u < units; u += gridDim.x) flags_region(a, u, bpb);
}

// Empty cooperative kernel: tells whether cooperative launches (with a
// programmatic dependency) are accepted, eagerly and in a captured graph.
__global__ void coop_probe_kernel() { pdl_enter(); }

// One block per 32 tiles (one word of tile bits); warp w scans tiles w, w+8,
// w+16, w+24 of the word.
__global__ void tile_bits_kernel(RemapArgs a, int ntiles) {
    pdl_enter();
    __shared__ uint32_t word;
    if (threadIdx.x == 0) word = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < 32; j += 8) {
        const int tile = blockIdx.x * 32 + j;
        if (tile >= ntiles) break;
        int lo = 0, hi = a.nlat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.lat[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
        }
        const LatDev &L = a.lat[lo];
        bool any = false;
        for (int c = lane; c < a.tile; c += 32) {
            const int idx = (tile - L.tile0) * a.tile + c;
            if (idx < L.n && a.flags[L.c_off + idx]) any = true;
        }
        if (__any_sync(0xffffffffu, any) && lane == 0) atomicOr(&word, 1u << j);
    }
    __syncthreads();
    if (threadIdx.x == 0) a.tbits[blockIdx.x] = word;
}

// ---------------------------------------------------------------------------
// whole-lattice kernels (creation, particle replacement, export)
// ---------------------------------------------------------------------------

__global__ void init_pid_kernel(const LatDev *lat, uint32_t *pid, uint32_t *pid_prev) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    uint32_t id = PID_FLUID;
    if (!L.py && j == 0)
        id = PID_WALL_YLO;
    else if (!L.py && j == L.ny - 1)
        id = PID_WALL_YHI;
    else if ((!L.px && (i == 0 || i == L.nx - 1)) || (!L.pz && (k == 0 || k == L.nz - 1)))
        id = PID_WALL;
    pid[L.c_off + x] = id;
    pid_prev[L.c_off + x] = PID_FLUID;
}

__global__ void flags_full_kernel(const LatDev *lat, uint8_t *flags, const uint32_t *pid, uint64_t *links,
                                  uint32_t *nbody) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    uint64_t lk;
    uint32_t p0;
    flags[L.c_off + x] = flag_of(L, pid, L.c_off, i, j, k, lk, p0);
    links[L.c_off + x] = lk;
    nbody[L.c_off + x] = p0;
}

__global__ void clear_particles_kernel(const LatDev *lat, uint8_t *flags, uint32_t *pid, uint32_t *pid_prev) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    const long long cg = L.c_off + x;
    const uint32_t id = pid[cg];
    if (id < PID_WALL) {
        pid_prev[cg] = id;
        pid[cg] = PID_FLUID;
        flags[cg] |= F_CHANGED;
    }
}

template <int PREC, int NEXT_ODD>
__global__ void fixup_full_kernel(RemapArgs a, const LatDev *lat) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    if (!(a.flags[L.c_off + x] & F_CHANGED)) return;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    fixup_cell<PREC, NEXT_ODD>(a, L, i, j, k, true);
}

template <int PREC, int NEXT_ODD>
__global__ void canonical_kernel(const LatDev *lat, const void *fv, const uint8_t *flags,
                                 const uint32_t *pid, double *rho, double *u3, uint8_t *fl_out,
                                 double *pdfs) {
    using S = Store<PREC>;
    using T = typename S::T;
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    const T *base = reinterpret_cast<const T *>(fv) + L.f_off;
    const long long np = L.npad, co = L.c_off;
    const uint8_t fl = flags[co + x];
    if (fl_out) fl_out[x] = (fl & F_WALL) ? LBM_FLAG_WALL : ((fl & F_SOLID) ? LBM_FLAG_PARTICLE : LBM_FLAG_FLUID);
    const int n = L.n;
    if (fl & F_SOLID) {
        if (rho) rho[x] = 0.0;
        if (u3) { u3[x] = 0.0; u3[n + x] = 0.0; u3[2 * n + x] = 0.0; }
        if (pdfs)
            for (int q = 0; q < Q; ++q) pdfs[(long long)q * n + x] = 0.0;
        return;
    }
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    double dr = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        double g;
        if (!NEXT_ODD) {
            g = (double)S::ld(base + q * np + x);
        } else {
            const int z = lin(L, i - cx(q), j - cy(q), k - cz(q));
            if ((flags[co + z] & (F_SOLID | F_FSLIP)) == F_SOLID)
                g = (double)S::ld(base + q * np + x);
            else
                g = (double)S::ld(base + opp(q) * np + z);
        }
        dr += g;
        jx += cx(q) * g;
        jy += cy(q) * g;
        jz += cz(q) * g;
        if (pdfs) pdfs[(long long)q * n + x] = g + wq(q) * L.rho0;
    }
    if (rho) rho[x] = L.rho0 + dr;
    if (u3) {
        u3[x] = jx / L.rho0 + 0.5 * L.g[0];
        u3[n + x] = jy / L.rho0 + 0.5 * L.g[1];
        u3[2 * n + x] = jz / L.rho0 + 0.5 * L.g[2];
    }
    (void)pid;
}

// Momentum stabilisation (Sec. 4.1): per block, the sum over its fluid cells
// of j = sum_q c_q f_q (offsets: sum_q c_q w_q rho0 = 0) as the coming sweep
// reads the populations (AA layout of parity NEXT_ODD, a solid neighbour's
// slot replaced by the cell's own, as in the export), and the number of fluid
// cells; FP64 atomics into acc[0..3], one set per block.
template <int PREC, int NEXT_ODD>
__global__ void __launch_bounds__(256) momentum_sum_kernel(const LatDev *lat, const void *fv,
                                                          const uint8_t *flags, double *acc) {
    pdl_enter();
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    const LatDev &L = *lat;
    const T *base = reinterpret_cast<const T *>(fv) + L.f_off;
    const long long np = L.npad, co = L.c_off;
    C sx = 0, sy = 0, sz = 0;
    int cnt = 0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < L.n; x += gridDim.x * blockDim.x) {
        const uint8_t fl = flags[co + x];
        if (fl & F_SOLID) continue;
        C jx = 0, jy = 0, jz = 0;
        if (!NEXT_ODD) {
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const C g = (C)S::ld(base + q * np + x);
                if (cx(q)) jx += cx(q) > 0 ? g : -g;
                if (cy(q)) jy += cy(q) > 0 ? g : -g;
                if (cz(q)) jz += cz(q) > 0 ? g : -g;
            }
        } else {
            const int yz = (int)L.divx.div((uint32_t)x), k = (int)L.divxy.div((uint32_t)x);
            const int i = x - yz * L.nx, j = yz - k * L.ny;
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const int z = lin(L, i - cx(q), j - cy(q), k - cz(q));
                const bool own = fl != 0 && (flags[co + z] & (F_SOLID | F_FSLIP)) == F_SOLID;
                const C g = (C)(own ? S::ld(base + q * np + x) : S::ld(base + opp(q) * np + z));
                if (cx(q)) jx += cx(q) > 0 ? g : -g;
                if (cy(q)) jy += cy(q) > 0 ? g : -g;
                if (cz(q)) jz += cz(q) > 0 ? g : -g;
            }
        }
        sx += jx;
        sy += jy;
        sz += jz;
        ++cnt;
    }
    double v[4] = {(double)sx, (double)sy, (double)sz, (double)cnt};
    __shared__ double part[8][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = warp_sum(v[c]);
    if (lane == 0)
        for (int c = 0; c < 4; ++c) part[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w][threadIdx.x];
        atomicAdd(acc + threadIdx.x, t);
    }
}

// Mean velocity from the sums: ubar = sum j / (rho0 N_fluid) into acc[4..6]
// and its FP32 copy; the sums are cleared for the next step.
__global__ void momentum_mean_kernel(const LatDev *lat, double *acc, float *accf) {
    pdl_enter();
    const int k = threadIdx.x;
    if (k >= 3) return;
    const double n = acc[3];
    const double u = n > 0.0 ? acc[k] / (lat->rho0 * n) : 0.0;
    acc[4 + k] = u;
    accf[k] = (float)u;
    __syncwarp(0x7u);
    acc[k] = 0.0;
    if (k == 0) acc[3] = 0.0;
}

template <int PREC, int NEXT_ODD>
__global__ void set_pdfs_kernel(const LatDev *lat, void *fv, const uint8_t *flags, const double *pdfs) {
    using S = Store<PREC>;
    using T = typename S::T;
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= L.n) return;
    T *base = reinterpret_cast<T *>(fv) + L.f_off;
    const long long np = L.npad, co = L.c_off;
    if (flags[co + x] & F_SOLID) return;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    const int n = L.n;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const double g = pdfs[(long long)q * n + x] - wq(q) * L.rho0;
        if (!NEXT_ODD) {
            S::st(base + q * np + x, (typename S::C)g);
        } else {
            const int z = lin(L, i - cx(q), j - cy(q), k - cz(q));
            if ((flags[co + z] & (F_SOLID | F_FSLIP)) == F_SOLID)
                S::st(base + q * np + x, (typename S::C)g);
            else
                S::st(base + opp(q) * np + z, (typename S::C)g);
        }
    }
}

// links: per-block counts, a single-block exclusive scan, then ordered writes
__device__ __forceinline__ uint32_t link_mask(const LatDev &L, const uint8_t *flags, int x) {
    const long long co = L.c_off;
    if (flags[co + x] & F_SOLID) return 0;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
    uint32_t m = 0;
#pragma unroll
    for (int q = 1; q < Q; ++q)
        if (flags[co + lin(L, i + cx(q), j + cy(q), k + cz(q))] & F_SOLID) m |= 1u << q;
    return m;
}

__global__ void link_count_kernel(const LatDev *lat, const uint8_t *flags, int *block_counts) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    int c = x < L.n ? __popc(link_mask(L, flags, x)) : 0;
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) block_counts[blockIdx.x] = v;
    }
}

__global__ void scan_kernel(int *counts, int nblocks, int *total) {
    // single block of 1024 threads: chunked exclusive scan
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nblocks ? counts[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblocks) counts[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += buf[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void link_write_kernel(const LatDev *lat, const uint8_t *flags, const uint32_t *pid,
                                  const int *block_offsets, int32_t *idx_out, int8_t *q_out,
                                  uint32_t *pid_out, int cap) {
    const LatDev &L = *lat;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t m = x < L.n ? link_mask(L, flags, x) : 0u;
    const int c = __popc(m);
    __shared__ int buf[1024];
    buf[threadIdx.x] = c;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int t = (int)threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += t;
        __syncthreads();
    }
    int pos = block_offsets[blockIdx.x] + buf[threadIdx.x] - c;
    if (!m) return;
    const int i = x % L.nx, j = (x / L.nx) % L.ny, k = x / (L.nx * L.ny);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (!((m >> q) & 1u)) continue;
        if (pos < cap) {
            if (idx_out) idx_out[pos] = x;
            if (q_out) q_out[pos] = (int8_t)q;
            if (pid_out) pid_out[pos] = pid[L.c_off + lin(L, i + cx(q), j + cy(q), k + cz(q))];
        }
        ++pos;
    }
}

template <int PREC>
cudaError_t remap_step_prec(int next_parity, const RemapArgs &a, int bpb, cudaStream_t s) {
    const unsigned grid = (unsigned)bpb * (unsigned)a.P.np;
    cudaError_t e;
    if (a.P.np == 1) {
        // one body: no cell can pass from one body to another, so uncover and
        // claim need no pass between them
        e = launch_pdl(remap_region_kernel<2>, grid, REMAP_BLOCK, 0, s, a, bpb);
    } else {
        e = launch_pdl(remap_region_kernel<0>, grid, REMAP_BLOCK, 0, s, a, bpb);
        if (e == cudaSuccess) e = launch_pdl(remap_region_kernel<1>, grid, REMAP_BLOCK, 0, s, a, bpb);
    }
    // the list passes: each thread strides over the list (its length is known
    // on the device only); the changed cells scale with the bodies, so the
    // grid is the region passes' (one box's blocks per body), at most about
    // one wave
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned wave = (unsigned)(sms > 0 ? sms : 1) * 8u;
    const unsigned lgrid = grid < wave ? grid : wave;
    if (e == cudaSuccess)
        e = next_parity ? launch_pdl(fixup_list_kernel<PREC, 1>, lgrid, REMAP_BLOCK, 0, s, a)
                        : launch_pdl(fixup_list_kernel<PREC, 0>, lgrid, REMAP_BLOCK, 0, s, a);
    if (e == cudaSuccess) e = launch_pdl(flags_list_kernel, lgrid, REMAP_BLOCK, 0, s, a);
    return e;
}

template <int PREC>
cudaError_t remap_fused_prec(int next_parity, const RemapArgs &a, int bpb, int grid, int mode, GridBar *bar,
                             cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(REMAP_BLOCK);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = mode == 2 ? 2 : 1;
    return next_parity ? cudaLaunchKernelEx(&cfg, remap_fused_kernel<PREC, 1>, a, bpb, bar)
                       : cudaLaunchKernelEx(&cfg, remap_fused_kernel<PREC, 0>, a, bpb, bar);
}

template <int PREC>
cudaError_t remap_full_prec(int next_parity, const RemapArgs &a, const LatDev &h, int li, cudaStream_t s) {
    const LatDev *d = a.lat + li;
    const int nb = (h.n + REMAP_BLOCK - 1) / REMAP_BLOCK;
    if (next_parity)
        fixup_full_kernel<PREC, 1><<<nb, REMAP_BLOCK, 0, s>>>(a, d);
    else
        fixup_full_kernel<PREC, 0><<<nb, REMAP_BLOCK, 0, s>>>(a, d);
    flags_full_kernel<<<nb, REMAP_BLOCK, 0, s>>>(d, a.flags, a.pid, a.links, a.nbody);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t canonical_prec(int next_parity, const LatDev &h, const LatDev *d, const void *f,
                           const uint8_t *flags, const uint32_t *pid, double *rho, double *u3,
                           uint8_t *fl, double *pdfs, cudaStream_t s) {
    const int nb = (h.n + 255) / 256;
    if (next_parity)
        canonical_kernel<PREC, 1><<<nb, 256, 0, s>>>(d, f, flags, pid, rho, u3, fl, pdfs);
    else
        canonical_kernel<PREC, 0><<<nb, 256, 0, s>>>(d, f, flags, pid, rho, u3, fl, pdfs);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t set_pdfs_prec(int next_parity, const LatDev &h, const LatDev *d, void *f,
                          const uint8_t *flags, const double *pdfs, cudaStream_t s) {
    const int nb = (h.n + 255) / 256;
    if (next_parity)
        set_pdfs_kernel<PREC, 1><<<nb, 256, 0, s>>>(d, f, flags, pdfs);
    else
        set_pdfs_kernel<PREC, 0><<<nb, 256, 0, s>>>(d, f, flags, pdfs);
    return cudaGetLastError();
}

}  // namespace

int kernels_per_remap_step(int np) { return np == 1 ? 3 : 4; }

int remap_fused_max_blocks() {
    int dev = 0, sms = 0, coop = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || sms <= 0) return 0;
    // every instantiation has the same launch bounds; the largest footprint decides
    int lo = 1 << 30;
    const void *ks[] = {(const void *)remap_fused_kernel<LBM_F64, 0>, (const void *)remap_fused_kernel<LBM_F64, 1>,
                        (const void *)remap_fused_kernel<LBM_F32, 0>, (const void *)remap_fused_kernel<LBM_F32, 1>,
                        (const void *)remap_fused_kernel<LBM_F16_OFFSET, 0>,
                        (const void *)remap_fused_kernel<LBM_F16_OFFSET, 1>,
                        (const void *)remap_fused_kernel<LBM_BF16_OFFSET, 0>,
                        (const void *)remap_fused_kernel<LBM_BF16_OFFSET, 1>};
    for (const void *k : ks) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, REMAP_BLOCK, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        lo = nb < lo ? nb : lo;
    }
    return lo > 0 ? lo * sms : 0;
}

int remap_fused_probe() {
    if (remap_fused_max_blocks() <= 0) return 0;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    auto launch = [&](int mode) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2);
        cfg.blockDim = dim3(32);
        cfg.stream = st;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = mode == 2 ? 2 : 1;
        return cudaLaunchKernelEx(&cfg, coop_probe_kernel);
    };
    // a cooperative launch between two ordinary programmatic launches, as in a step
    auto sequence = [&](int mode) {
        cudaError_t e = launch_pdl(coop_probe_kernel, 1, 32, 0, st);
        if (e == cudaSuccess) e = launch(mode);
        if (e == cudaSuccess) e = launch_pdl(coop_probe_kernel, 1, 32, 0, st);
        return e;
    };
    int best = 0;
    for (int mode = 2; mode >= 1 && !best; --mode) {
        cudaError_t e = sequence(mode);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t x = nullptr;
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t el = sequence(mode);
                e = cudaStreamEndCapture(st, &g);
                if (e == cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(x, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (x) cudaGraphExecDestroy(x);
            if (g) cudaGraphDestroy(g);
        }
        if (e == cudaSuccess) best = mode;
        cudaGetLastError();
    }
    cudaStreamDestroy(st);
    return best;
}

cudaError_t launch_tile_bits(const RemapArgs &a, int ntiles, cudaStream_t s) {
    if (!a.tbits || ntiles <= 0) return cudaSuccess;
    return launch_pdl(tile_bits_kernel, (ntiles + 31) / 32, 256, 0, s, a, ntiles);
}

cudaError_t launch_rigid_body(const RemapArgs &a, cudaStream_t s) {
    const int n = a.P.np + a.nlat;  // one warp per body, then one per lattice
    if (n <= 0) return cudaSuccess;
    return launch_pdl(rigid_body_kernel, (int)((32ll * n + 127) / 128), 128, 0, s, a);
}

#define LBM_DISPATCH(prec, call)                                        \
    switch (prec) {                                                     \
    case LBM_F64: return call<LBM_F64>;                                 \
    case LBM_F32: return call<LBM_F32>;                                 \
    case LBM_F16_OFFSET: return call<LBM_F16_OFFSET>;                   \
    case LBM_BF16_OFFSET: return call<LBM_BF16_OFFSET>;                 \
    }                                                                   \
    return cudaErrorInvalidValue;

cudaError_t launch_remap_step(int prec, int next_parity, const RemapArgs &a, int bpb, cudaStream_t s) {
    if (a.P.np <= 0) return cudaSuccess;
    switch (prec) {
    case LBM_F64: return remap_step_prec<LBM_F64>(next_parity, a, bpb, s);
    case LBM_F32: return remap_step_prec<LBM_F32>(next_parity, a, bpb, s);
    case LBM_F16_OFFSET: return remap_step_prec<LBM_F16_OFFSET>(next_parity, a, bpb, s);
    case LBM_BF16_OFFSET: return remap_step_prec<LBM_BF16_OFFSET>(next_parity, a, bpb, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_remap_fused(int prec, int next_parity, const RemapArgs &a, int bpb, int grid, int mode,
                               GridBar *bar, cudaStream_t s) {
    if (a.P.np <= 0 || grid <= 0 || mode <= 0) return cudaErrorInvalidValue;
    switch (prec) {
    case LBM_F64: return remap_fused_prec<LBM_F64>(next_parity, a, bpb, grid, mode, bar, s);
    case LBM_F32: return remap_fused_prec<LBM_F32>(next_parity, a, bpb, grid, mode, bar, s);
    case LBM_F16_OFFSET: return remap_fused_prec<LBM_F16_OFFSET>(next_parity, a, bpb, grid, mode, bar, s);
    case LBM_BF16_OFFSET: return remap_fused_prec<LBM_BF16_OFFSET>(next_parity, a, bpb, grid, mode, bar, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_momentum_mean(int prec, int next_parity, const LatDev &h, const LatDev *d, const void *f,
                                 const uint8_t *flags, double *acc, float *accf, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = ((long long)h.n + 255) / 256;
    const int grid = (int)(want < 4ll * sms ? want : 4ll * sms);
    cudaError_t e = cudaErrorInvalidValue;
#define LBM_MOMENTUM(P)                                                                              \
    e = next_parity ? launch_pdl(momentum_sum_kernel<P, 1>, grid, 256, 0, s, d, f, flags, acc)        \
                    : launch_pdl(momentum_sum_kernel<P, 0>, grid, 256, 0, s, d, f, flags, acc);
    switch (prec) {
    case LBM_F64: LBM_MOMENTUM(LBM_F64) break;
    case LBM_F32: LBM_MOMENTUM(LBM_F32) break;
    case LBM_F16_OFFSET: LBM_MOMENTUM(LBM_F16_OFFSET) break;
    case LBM_BF16_OFFSET: LBM_MOMENTUM(LBM_BF16_OFFSET) break;
    }
#undef LBM_MOMENTUM
    if (e != cudaSuccess) return e;
    return launch_pdl(momentum_mean_kernel, 1, 32, 0, s, d, acc, accf);
}

// Full re-map for a new particle set, in three launches: clear the particle
// cells of each lattice, claim from the new poses (regions computed on the
// host), then fix up populations and flags of each lattice.
cudaError_t launch_clear_particles(const LatDev &h, const RemapArgs &a, int li, cudaStream_t s) {
    const int nb = (h.n + REMAP_BLOCK - 1) / REMAP_BLOCK;
    clear_particles_kernel<<<nb, REMAP_BLOCK, 0, s>>>(a.lat + li, a.flags, a.pid, a.pid_prev);
    return cudaGetLastError();
}

cudaError_t launch_claim_all(const RemapArgs &a, int blocks_per_body, cudaStream_t s) {
    if (a.P.np <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)blocks_per_body * (unsigned)a.P.np;
    remap_region_kernel<1><<<grid, REMAP_BLOCK, 0, s>>>(a, blocks_per_body);
    return cudaGetLastError();
}

cudaError_t launch_remap_full(int prec, int next_parity, const RemapArgs &a, const LatDev &h, int li,
                              cudaStream_t s) {
    switch (prec) {
    case LBM_F64: return remap_full_prec<LBM_F64>(next_parity, a, h, li, s);
    case LBM_F32: return remap_full_prec<LBM_F32>(next_parity, a, h, li, s);
    case LBM_F16_OFFSET: return remap_full_prec<LBM_F16_OFFSET>(next_parity, a, h, li, s);
    case LBM_BF16_OFFSET: return remap_full_prec<LBM_BF16_OFFSET>(next_parity, a, h, li, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init_cells(const LatDev &h, const LatDev *d, uint8_t *flags, uint32_t *pid,
                              uint32_t *pid_prev, uint64_t *links, uint32_t *nbody, cudaStream_t s) {
    const int nb = (h.n + 255) / 256;
    init_pid_kernel<<<nb, 256, 0, s>>>(d, pid, pid_prev);
    flags_full_kernel<<<nb, 256, 0, s>>>(d, flags, pid, links, nbody);
    return cudaGetLastError();
}

cudaError_t launch_canonical(int prec, int next_parity, const LatDev &h, const LatDev *d, const void *f,
                             const uint8_t *flags, const uint32_t *pid, double *rho, double *u3,
                             uint8_t *fl, double *pdfs, cudaStream_t s) {
    switch (prec) {
    case LBM_F64: return canonical_prec<LBM_F64>(next_parity, h, d, f, flags, pid, rho, u3, fl, pdfs, s);
    case LBM_F32: return canonical_prec<LBM_F32>(next_parity, h, d, f, flags, pid, rho, u3, fl, pdfs, s);
    case LBM_F16_OFFSET:
        return canonical_prec<LBM_F16_OFFSET>(next_parity, h, d, f, flags, pid, rho, u3, fl, pdfs, s);
    case LBM_BF16_OFFSET:
        return canonical_prec<LBM_BF16_OFFSET>(next_parity, h, d, f, flags, pid, rho, u3, fl, pdfs, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_set_pdfs(int prec, int next_parity, const LatDev &h, const LatDev *d, void *f,
                            const uint8_t *flags, const double *pdfs, cudaStream_t s) {
    switch (prec) {
    case LBM_F64: return set_pdfs_prec<LBM_F64>(next_parity, h, d, f, flags, pdfs, s);
    case LBM_F32: return set_pdfs_prec<LBM_F32>(next_parity, h, d, f, flags, pdfs, s);
    case LBM_F16_OFFSET: return set_pdfs_prec<LBM_F16_OFFSET>(next_parity, h, d, f, flags, pdfs, s);
    case LBM_BF16_OFFSET: return set_pdfs_prec<LBM_BF16_OFFSET>(next_parity, h, d, f, flags, pdfs, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_links(const LatDev &h, const LatDev *d, const uint8_t *flags, const uint32_t *pid,
                         int *block_counts, int nblocks, int32_t *idx, int8_t *q, uint32_t *pid_out,
                         int cap, int *total, cudaStream_t s) {
    link_count_kernel<<<nblocks, 256, 0, s>>>(d, flags, block_counts);
    scan_kernel<<<1, 1024, 0, s>>>(block_counts, nblocks, total);
    link_write_kernel<<<nblocks, 256, 0, s>>>(d, flags, pid, block_counts, idx, q, pid_out, cap);
    return cudaGetLastError();
}

}  // namespace lbm
