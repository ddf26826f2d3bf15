// lbm_closure.cu -- learned force/torque closure: per-body flow features,
// a 86-64-64-64-6 ReLU network on the FP16 tensor cores (FP32 accumulation)
// for inference inside the time step and for training (forward, backward,
// Adam).  The network adds a correction to the momentum-exchange force and
// torque (Eqs. TransferredMomentum, LBMhydrodynForce) before the rigid-body
// update (Sec. 4.3); the paper has no closure, so the feature set, the scales
// and the network follow the readings stated with each function.
//
// Tensor-core step: mma.sync.m16n8k16 (FP16 A and B, FP32 C/D).  The
// network is tiny (~14 k multiply-adds per body), so each warp owns 16 rows
// (bodies or samples) and walks the 8-column tiles of every layer with its
// operands in shared memory.
#include <cmath>
#include <mutex>

#include "lbm_internal.cuh"

namespace lbm {

namespace {

constexpr int NIN = CL_IN, NINP = 96, NH = CL_HID, NOUT = CL_OUT, NOUTP = 16;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NOUT * NH, NPAR = OB4 + NOUT;
static_assert(NPAR == CL_PARAMS, "closure parameter layout");

constexpr int ROWS = 128;  // rows (bodies or samples) per pass of a block: 8 warps x 16

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ uint32_t pack2(__half lo, __half hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

// D = A B + D on one 16x8 tile (PTX ISA fragment layouts of m16n8k16 .f16).
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A matrix in shared memory: element (r, c) at p[r * ld + c], or at
// p[c * ld + r] when transposed.
struct SMat {
    const __half *p;
    int ld;
    bool tr;
    __device__ __forceinline__ __half at(int r, int c) const { return tr ? p[c * ld + r] : p[r * ld + c]; }
};

// c += A(m0 .. m0+15, 0 .. K-1) B(0 .. K-1, n0 .. n0+7), K a multiple of 16.
// Thread (g = lane/4, t = lane%4) ends with c[0], c[1] at row m0+g, columns
// n0+2t, n0+2t+1, and c[2], c[3] at row m0+g+8.
__device__ __forceinline__ void tile_mma(float (&c)[4], const SMat &A, int m0, const SMat &B, int n0, int K) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4], b[2];
        const int ka = k0 + 2 * t;
        a[0] = pack2(A.at(m0 + g, ka), A.at(m0 + g, ka + 1));
        a[1] = pack2(A.at(m0 + g + 8, ka), A.at(m0 + g + 8, ka + 1));
        a[2] = pack2(A.at(m0 + g, ka + 8), A.at(m0 + g, ka + 9));
        a[3] = pack2(A.at(m0 + g + 8, ka + 8), A.at(m0 + g + 8, ka + 9));
        b[0] = pack2(B.at(ka, n0 + g), B.at(ka + 1, n0 + g));
        b[1] = pack2(B.at(ka + 8, n0 + g), B.at(ka + 9, n0 + g));
        mma16816(c, a, b);
    }
}

// The same product when A is row-major (a[r][k] at A + r lda + k) and B is
// stored as its transpose, B(k, n) at Bt + n ldb + k (a layer's weights
// [out][in]): the fragments come straight from shared memory with ldmatrix
// (four 8x8 matrices of A, two of B per 16-wide k step; lane l gives the
// address of row l % 8 of matrix l / 8), whose register layout is the
// m16n8k16 fragment layout.  Rows must start on 16 bytes (lda, ldb multiples
// of 8 halves, 16-byte aligned bases).
__device__ __forceinline__ void tile_mma_ldm(float (&c)[4], const __half *A, int lda, int m0, const __half *Bt,
                                             int ldb, int n0, int K) {
    const int lane = threadIdx.x & 31;
    const int mat = lane >> 3, row = lane & 7;
    // A: matrices (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15)
    const __half *pa = A + (m0 + row + 8 * (mat & 1)) * lda + 8 * (mat >> 1);
    // B: matrices (n 0-7, k 0-7), (n 0-7, k 8-15); lanes 16-31 repeat lanes 0-15
    const __half *pb = Bt + (n0 + row) * ldb + 8 * (mat & 1);
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4], b[2];
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                     : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                     : "r"((uint32_t)__cvta_generic_to_shared(pa + k0)));
        asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                     : "=r"(b[0]), "=r"(b[1])
                     : "r"((uint32_t)__cvta_generic_to_shared(pb + k0)));
        mma16816(c, a, b);
    }
}

// Shared-memory image of the network: FP16 weights zero-padded to the tile
// grid ([out][in] rows, W1 to 96 inputs, W4 to 16 outputs), FP32 biases.
struct NetSmem {
    __half w1[NH * NINP], w2[NH * NH], w3[NH * NH], w4[NOUTP * NH];
    float b1[NH], b2[NH], b3[NH], b4[NOUTP];
};

__device__ void load_net(NetSmem &s, const __half *par) {
    for (int i = threadIdx.x; i < NH * NINP; i += blockDim.x) {
        const int o = i / NINP, c = i % NINP;
        s.w1[i] = c < NIN ? par[OW1 + o * NIN + c] : __float2half(0.f);
    }
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
        s.w2[i] = par[OW2 + i];
        s.w3[i] = par[OW3 + i];
    }
    for (int i = threadIdx.x; i < NOUTP * NH; i += blockDim.x)
        s.w4[i] = i < NOUT * NH ? par[OW4 + i] : __float2half(0.f);
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        s.b1[i] = __half2float(par[OB1 + i]);
        s.b2[i] = __half2float(par[OB2 + i]);
        s.b3[i] = __half2float(par[OB3 + i]);
    }
    for (int i = threadIdx.x; i < NOUTP; i += blockDim.x) s.b4[i] = i < NOUT ? __half2float(par[OB4 + i]) : 0.f;
}

// One dense layer for this warp's 16 rows: out = act(in W^T + b) stored in
// FP16 (ReLU for hidden layers), or the FP32 output tile for the last layer.
template <bool RELU>
__device__ __forceinline__ void dense(const __half *in, int ldin, int K, const __half *w, int ldw,
                                      const float *bias, int N, __half *out, int ldout, int m0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int n0 = 0; n0 < N; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile_mma_ldm(c, in, ldin, m0, w, ldw, n0, K);
        const int col = n0 + 2 * t;
        float v[4] = {c[0] + bias[col], c[1] + bias[col + 1], c[2] + bias[col], c[3] + bias[col + 1]};
        if (RELU)
            for (int k = 0; k < 4; ++k) v[k] = fmaxf(v[k], 0.f);
        *reinterpret_cast<__half2 *>(out + (m0 + g) * ldout + col) = __floats2half2_rn(v[0], v[1]);
        *reinterpret_cast<__half2 *>(out + (m0 + g + 8) * ldout + col) = __floats2half2_rn(v[2], v[3]);
    }
}

// Forward pass of this warp's 16 rows of X (96 padded FP16 inputs per row);
// h1..h3 receive the hidden activations; the 16 x 8 output tile is returned
// in c (columns 0..5 meaningful).
__device__ __forceinline__ void forward_rows(const NetSmem &s, const __half *X, __half *h1, __half *h2,
                                             __half *h3, int m0, float (&c)[4]) {
    dense<true>(X, NINP, NINP, s.w1, NINP, s.b1, NH, h1, NH, m0);
    __syncwarp();
    dense<true>(h1, NH, NH, s.w2, NH, s.b2, NH, h2, NH, m0);
    __syncwarp();
    dense<true>(h2, NH, NH, s.w3, NH, s.b3, NH, h3, NH, m0);
    __syncwarp();
    const int t = threadIdx.x & 3;
    c[0] = c[1] = c[2] = c[3] = 0.f;
    tile_mma_ldm(c, h3, NH, m0, s.w4, NH, 0, NH);
    c[0] += s.b4[2 * t];
    c[1] += s.b4[2 * t + 1];
    c[2] += s.b4[2 * t];
    c[3] += s.b4[2 * t + 1];
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------

// Velocity of cell x as the fields export reports it (sum c g / rho0 + g/2 on
// fluid cells, zero on wall and particle cells), reading the populations in
// the AA layout the next sweep (parity NEXT_ODD) expects.
template <int PREC, int NEXT_ODD>
__device__ __forceinline__ void cell_velocity(const LatDev &L, const void *fv, const uint8_t *flags, int i, int j,
                                              int k, float u[3]) {
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;  // FP64 only on FP64 lattices (GB300's FP64 rate is low)
    u[0] = u[1] = u[2] = 0.f;
    const int x = i + L.nx * (j + L.ny * k);
    if (flags[L.c_off + x] & F_SOLID) return;
    const T *base = reinterpret_cast<const T *>(fv) + L.f_off;
    const long long np = L.npad;
    C jx = 0, jy = 0, jz = 0;
    // odd layout: the neighbours' flag bytes first (all in flight together),
    // then the populations they select
    const T *src[Q];
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (!NEXT_ODD) {
            src[q] = base + q * np + x;
        } else {
            const int zi = wrapi(i - cx(q), L.nx), zj = wrapi(j - cy(q), L.ny), zk = wrapi(k - cz(q), L.nz);
            const int z = zi + L.nx * (zj + L.ny * zk);
            src[q] = (flags[L.c_off + z] & (F_SOLID | F_FSLIP)) == F_SOLID ? base + q * np + x
                                                                           : base + opp(q) * np + z;
        }
    }
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        const C g = S::ld(src[q]);
        if (cx(q)) jx += cx(q) > 0 ? g : -g;
        if (cy(q)) jy += cy(q) > 0 ? g : -g;
        if (cz(q)) jz += cz(q) > 0 ? g : -g;
    }
    const LatPar<C> lp(L);
    u[0] = (float)(jx * lp.inv_rho0 + C(0.5) * lp.g[0]);
    u[1] = (float)(jy * lp.inv_rho0 + C(0.5) * lp.g[1]);
    u[2] = (float)(jz * lp.inv_rho0 + C(0.5) * lp.g[2]);
}

// One block of FEAT_THREADS threads per body: thread t < 216 takes corner
// t % 8 of sample point s = t / 8 (offsets (1.5 a i, 1.5 b j, 1.5 c k),
// s = 9(i+1) + 3(j+1) + (k+1)), the cell of that corner of the point's
// surrounding cube (periodic axes wrap, the others clamp) and its trilinear
// weight; the eight corners of a point are eight consecutive lanes and sum
// their weighted velocities by shuffles.  The corner-0 lane subtracts the
// body's rigid motion continued to the point (U + Omega x R o_s), rotates
// into the body frame and scales by 1/(shear rate * a); threads 216 and 217
// write the body axis, a/b and b.  A corner per thread keeps eight times as
// many cell reads in flight as a point per thread.
constexpr int FEAT_THREADS = 224;

template <int PREC, int NEXT_ODD>
__global__ void __launch_bounds__(FEAT_THREADS) closure_features_kernel(ClosureArgs a) {
    pdl_enter();
    const int p = (int)blockIdx.x;
    const int t = (int)threadIdx.x;
    const PartDev &P = a.P;
    if (p >= P.np) return;  // uniform per block
    const LatDev &L = a.lat[P.cell[p]];
    const float *bf = P.bodyf + BF_STRIDE * (size_t)p;
    float R[9], pos[3];
    for (int k = 0; k < 9; ++k) R[k] = bf[BF_R + k];
    for (int k = 0; k < 3; ++k) pos[k] = bf[BF_POS + k] + bf[BF_POSLO + k];
    const float sa = (float)P.semi[3 * (size_t)p], sb = (float)P.semi[3 * (size_t)p + 1],
                sc = (float)P.semi[3 * (size_t)p + 2];
    float *out = a.feat + (size_t)p * NIN;
    const int s = t >> 3, corner = t & 7;
    float ro[3] = {0.f, 0.f, 0.f}, u[3] = {0.f, 0.f, 0.f};
    if (s < 27) {
        const int i = s / 9 - 1, j = (s / 3) % 3 - 1, k = s % 3 - 1;
        const float o[3] = {1.5f * sa * i, 1.5f * sb * j, 1.5f * sc * k};
        float x[3];
        for (int r = 0; r < 3; ++r) {
            ro[r] = R[3 * r] * o[0] + R[3 * r + 1] * o[1] + R[3 * r + 2] * o[2];
            x[r] = pos[r] + ro[r];
        }
        const int dims[3] = {L.nx, L.ny, L.nz}, per[3] = {L.px, L.py, L.pz};
        int idx[3];
        float w = 1.f;
        for (int r = 0; r < 3; ++r) {
            const float fl = floorf(x[r]);
            const float w1 = x[r] - fl;
            const int off = (corner >> r) & 1;
            w *= off ? w1 : 1.f - w1;
            int v = (int)fl + off;
            if (per[r]) {
                v %= dims[r];
                if (v < 0) v += dims[r];
            } else {
                v = min(max(v, 0), dims[r] - 1);
            }
            idx[r] = v;
        }
        float uc[3];
        cell_velocity<PREC, NEXT_ODD>(L, a.f, a.flags, idx[0], idx[1], idx[2], uc);
        for (int r = 0; r < 3; ++r) u[r] = w * uc[r];
    }
    // corners 0..7 of a point are lanes 8m .. 8m+7 of one warp: a butterfly
    // over them sums the eight weighted velocities (pairwise, in FP32)
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
        for (int r = 0; r < 3; ++r) u[r] += __shfl_xor_sync(0xffffffffu, u[r], o);
    if (s < 27 && corner == 0) {
        float U[3], W[3];
        for (int k = 0; k < 3; ++k) {
            U[k] = bf[BF_U + k];
            W[k] = bf[BF_W + k];
        }
        const float V = L.cl_gamma > 0.f ? L.cl_gamma * sa : 1.f;
        // relative to the rigid motion continued to the sample point
        const float d[3] = {u[0] - (U[0] + (W[1] * ro[2] - W[2] * ro[1])),
                            u[1] - (U[1] + (W[2] * ro[0] - W[0] * ro[2])),
                            u[2] - (U[2] + (W[0] * ro[1] - W[1] * ro[0]))};
        for (int r = 0; r < 3; ++r) out[3 * s + r] = (R[r] * d[0] + R[3 + r] * d[1] + R[6 + r] * d[2]) / V;
    } else if (t == 216) {
        out[81] = R[0];
        out[82] = R[3];
        out[83] = R[6];
    } else if (t == 217) {
        out[84] = sa / sb;
        out[85] = sb;
    }
}

// ---------------------------------------------------------------------------
// inference
// ---------------------------------------------------------------------------

struct InferSmem {
    NetSmem net;
    __half x[ROWS * NINP];
    __half h1[ROWS * NH], h2[ROWS * NH], h3[ROWS * NH];
};
// ldmatrix reads rows of 16 bytes: every array starts on 16 bytes
static_assert(sizeof(NetSmem) % 16 == 0 && (ROWS * NINP * 2) % 16 == 0 && (ROWS * NH * 2) % 16 == 0,
              "16-byte aligned shared-memory operands");

// Block of 8 warps, 128 rows.  APPLY: rows are bodies; their outputs become
// the world-frame correction R dF * mu*gamma*a*b, R dM * mu*gamma*a^2*b, added
// into accumulator copy 0 of the body (summed with the sweep's copies by the
// rigid-body update).  Otherwise the FP32 outputs go to y (n x 6).
template <bool APPLY>
__global__ void __launch_bounds__(256) mlp_infer_kernel(MlpArgs m, ClosureArgs a) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &s = *reinterpret_cast<InferSmem *>(smem_raw);
    load_net(s.net, m.par16);
    const int row0 = blockIdx.x * ROWS;
    for (int i = threadIdx.x; i < ROWS * NINP; i += blockDim.x) {
        const int r = i / NINP, c = i % NINP;
        const float v = (row0 + r < m.n && c < NIN) ? m.x[(size_t)(row0 + r) * NIN + c] : 0.f;
        s.x[i] = __float2half(v);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16;
    float c[4];
    forward_rows(s.net, s.x, s.h1, s.h2, s.h3, m0, c);
    // outputs of rows m0+g (c0, c1) and m0+g+8 (c2, c3), columns 2t, 2t+1
    __shared__ float o[ROWS][8];
    o[m0 + g][2 * t] = c[0];
    o[m0 + g][2 * t + 1] = c[1];
    o[m0 + g + 8][2 * t] = c[2];
    o[m0 + g + 8][2 * t + 1] = c[3];
    __syncthreads();
    const int r = threadIdx.x;
    if (r >= ROWS || row0 + r >= m.n) return;
    const int p = row0 + r;
    if (!APPLY) {
        for (int k = 0; k < NOUT; ++k) m.out[(size_t)p * NOUT + k] = o[r][k];
        return;
    }
    const PartDev &P = a.P;
    const LatDev &L = a.lat[P.cell[p]];
    if (!(L.cl_gamma > 0.f)) return;
    const float *bf = P.bodyf + BF_STRIDE * (size_t)p;
    const double sa = P.semi[3 * (size_t)p], sb = P.semi[3 * (size_t)p + 1];
    const double fs = (double)L.cl_mu * L.cl_gamma * sa * sb, ms = fs * sa;
    double *acc = P.acc + 6 * ((size_t)p * ACC_COPIES);
    for (int r2 = 0; r2 < 3; ++r2) {
        const double dF = (double)bf[BF_R + 3 * r2] * o[r][0] + (double)bf[BF_R + 3 * r2 + 1] * o[r][1] +
                          (double)bf[BF_R + 3 * r2 + 2] * o[r][2];
        const double dM = (double)bf[BF_R + 3 * r2] * o[r][3] + (double)bf[BF_R + 3 * r2 + 1] * o[r][4] +
                          (double)bf[BF_R + 3 * r2 + 2] * o[r][5];
        atomicAdd(acc + r2, dF * fs);
        atomicAdd(acc + 3 + r2, dM * ms);
    }
}

// ---------------------------------------------------------------------------
// training: one block computes loss and gradient over the whole batch in
// passes of 128 rows; Adam updates the FP32 master parameters
// ---------------------------------------------------------------------------

struct TrainSmem {
    NetSmem net;
    __half x[ROWS * NINP];
    __half h1[ROWS * NH], h2[ROWS * NH], h3[ROWS * NH];
    __half d_o[ROWS * NOUTP];             // dL/d(output) without the 2/(n*6) factor
    __half da[ROWS * NH], db[ROWS * NH];  // back-propagated deltas (ping-pong)
    float red[256];
};

// grad(W)[out][in] += sum over the 128 rows of dlt[row][out] * act[row][in]
// for the tiles of this warp; the tile grid is M_pad x N (16 x 8 tiles).
__device__ void weight_grad(const __half *dlt, int ld_d, int M, int Mstore, const __half *act, int ld_a,
                            int N, int Nstore, float *g, int ldg) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane >> 2, t = lane & 3;
    const int mt = M / 16, nt = N / 8;
    const SMat A{dlt, ld_d, true}, B{act, ld_a, false};
    for (int tile = warp; tile < mt * nt; tile += 8) {
        const int m0 = (tile / nt) * 16, n0 = (tile % nt) * 8;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile_mma(c, A, m0, B, n0, ROWS);
        const int rr[4] = {m0 + gi, m0 + gi, m0 + gi + 8, m0 + gi + 8};
        const int cc[4] = {n0 + 2 * t, n0 + 2 * t + 1, n0 + 2 * t, n0 + 2 * t + 1};
        for (int k = 0; k < 4; ++k)
            if (rr[k] < Mstore && cc[k] < Nstore) g[rr[k] * ldg + cc[k]] += c[k];
    }
}

// delta_below[row][in] = (sum_out dlt[row][out] W[out][in]) * (act[row][in] > 0)
__device__ void back_delta(const __half *dlt, int ld_d, int K, const __half *w, int ldw, const __half *act,
                           int N, __half *out, int m0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const SMat A{dlt, ld_d, false}, B{w, ldw, false};
    for (int n0 = 0; n0 < N; n0 += 8) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        tile_mma(c, A, m0, B, n0, K);
        const int col = n0 + 2 * t;
        const int rr[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
        const int cc[4] = {col, col + 1, col, col + 1};
        for (int k = 0; k < 4; ++k) {
            const bool on = __half2float(act[rr[k] * NH + cc[k]]) > 0.f;
            out[rr[k] * NH + cc[k]] = __float2half(on ? c[k] : 0.f);
        }
    }
}

__device__ void bias_grad(const __half *dlt, int ld_d, int N, int Nstore, float *g) {
    for (int col = threadIdx.x; col < N; col += blockDim.x) {
        if (col >= Nstore) continue;
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += __half2float(dlt[r * ld_d + col]);
        g[col] += s;
    }
}

__global__ void __launch_bounds__(256) mlp_grad_kernel(MlpArgs m) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(smem_raw);
    float *grad = m.grad;
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) grad[i] = 0.f;
    load_net(s.net, m.par16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16;
    float lsum = 0.f;
    __syncthreads();
    for (int row0 = 0; row0 < m.n; row0 += ROWS) {
        for (int i = threadIdx.x; i < ROWS * NINP; i += blockDim.x) {
            const int r = i / NINP, c = i % NINP;
            const float v = (row0 + r < m.n && c < NIN) ? m.x[(size_t)(row0 + r) * NIN + c] : 0.f;
            s.x[i] = __float2half(v);
        }
        __syncthreads();
        float c[4];
        forward_rows(s.net, s.x, s.h1, s.h2, s.h3, m0, c);
        // output delta (o - y) on valid rows and the six outputs, zero elsewhere
        const int rr[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
        const int cc[4] = {2 * t, 2 * t + 1, 2 * t, 2 * t + 1};
        for (int k = 0; k < 4; ++k) {
            const int row = row0 + rr[k];
            float d = 0.f;
            if (row < m.n && cc[k] < NOUT) {
                d = c[k] - m.y[(size_t)row * NOUT + cc[k]];
                lsum += d * d;
            }
            s.d_o[rr[k] * NOUTP + cc[k]] = __float2half(d);
        }
        for (int k = 8; k < NOUTP; ++k)
            if (lane < 16) s.d_o[(m0 + lane) * NOUTP + k] = __float2half(0.f);
        __syncthreads();
        // layer 4
        weight_grad(s.d_o, NOUTP, 16, NOUT, s.h3, NH, NH, NH, grad + OW4, NH);
        bias_grad(s.d_o, NOUTP, NOUTP, NOUT, grad + OB4);
        back_delta(s.d_o, NOUTP, NOUTP, s.net.w4, NH, s.h3, NH, s.da, m0);
        __syncthreads();
        // layer 3
        weight_grad(s.da, NH, NH, NH, s.h2, NH, NH, NH, grad + OW3, NH);
        bias_grad(s.da, NH, NH, NH, grad + OB3);
        back_delta(s.da, NH, NH, s.net.w3, NH, s.h2, NH, s.db, m0);
        __syncthreads();
        // layer 2
        weight_grad(s.db, NH, NH, NH, s.h1, NH, NH, NH, grad + OW2, NH);
        bias_grad(s.db, NH, NH, NH, grad + OB2);
        back_delta(s.db, NH, NH, s.net.w2, NH, s.h1, NH, s.da, m0);
        __syncthreads();
        // layer 1 (inputs padded to 96 columns, 86 stored)
        weight_grad(s.da, NH, NH, NH, s.x, NINP, NINP, NIN, grad + OW1, NIN);
        bias_grad(s.da, NH, NH, NH, grad + OB1);
        __syncthreads();
    }
    // d(mean squared error) = 2 (o - y) / (n * 6)
    const float scale = 2.f / ((float)m.n * NOUT);
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) grad[i] *= scale;
    s.red[threadIdx.x] = lsum;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s.red[threadIdx.x] += s.red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && m.loss) *m.loss = s.red[0] / ((float)m.n * NOUT);
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters; c1 = 1 - beta1^t,
// c2 = 1 - beta2^t; refreshes the FP16 working copy.
__global__ void adam_kernel(MlpArgs m, float lr, float beta1, float beta2, float eps, float c1, float c2) {
    pdl_enter();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float gr = m.grad[i];
    const float mi = beta1 * m.adam_m[i] + (1.f - beta1) * gr;
    const float vi = beta2 * m.adam_v[i] + (1.f - beta2) * gr * gr;
    m.adam_m[i] = mi;
    m.adam_v[i] = vi;
    const float p = m.par32[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    m.par32[i] = p;
    m.par16[i] = __float2half(p);
}

__global__ void to_half_kernel(const float *src, __half *dst, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2half(src[i]);
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// The dynamic shared memory limit is a per-device attribute of a kernel:
// raised once per device (done[d]), under one mutex (launches come from any
// host thread, each context on its own device).
constexpr int SMEM_MAX_DEVICES = 64;
inline std::mutex &smem_mu() {
    static std::mutex m;
    return m;
}
template <class K>
cudaError_t set_smem_once(K kernel, size_t bytes, bool (&done)[SMEM_MAX_DEVICES]) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= SMEM_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(smem_mu());
    if (!done[dev]) {
        if ((e = set_smem(kernel, bytes)) != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

template <int PREC>
cudaError_t features_prec(int next_odd, const ClosureArgs &a, int np, cudaStream_t s) {
    return next_odd ? launch_pdl(closure_features_kernel<PREC, 1>, np, FEAT_THREADS, 0, s, a)
                    : launch_pdl(closure_features_kernel<PREC, 0>, np, FEAT_THREADS, 0, s, a);
}

}  // namespace

int closure_param_count() { return NPAR; }

cudaError_t launch_closure_features(int prec, int next_odd, const ClosureArgs &a, cudaStream_t s) {
    if (a.P.np <= 0) return cudaSuccess;
    switch (prec) {
    case LBM_F64: return features_prec<LBM_F64>(next_odd, a, a.P.np, s);
    case LBM_F32: return features_prec<LBM_F32>(next_odd, a, a.P.np, s);
    case LBM_F16_OFFSET: return features_prec<LBM_F16_OFFSET>(next_odd, a, a.P.np, s);
    case LBM_BF16_OFFSET: return features_prec<LBM_BF16_OFFSET>(next_odd, a, a.P.np, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_mlp_infer(const MlpArgs &m, const ClosureArgs *apply, cudaStream_t s) {
    if (m.n <= 0) return cudaSuccess;
    const size_t smem = sizeof(InferSmem);
    const int blocks = (m.n + ROWS - 1) / ROWS;
    cudaError_t e;
    if (apply) {
        static bool attr[SMEM_MAX_DEVICES] = {};
        if ((e = set_smem_once(mlp_infer_kernel<true>, smem, attr)) != cudaSuccess) return e;
        return launch_pdl(mlp_infer_kernel<true>, blocks, 256, smem, s, m, *apply);
    }
    static bool attr[SMEM_MAX_DEVICES] = {};
    if ((e = set_smem_once(mlp_infer_kernel<false>, smem, attr)) != cudaSuccess) return e;
    return launch_pdl(mlp_infer_kernel<false>, blocks, 256, smem, s, m, ClosureArgs{});
}

cudaError_t launch_mlp_grad(const MlpArgs &m, cudaStream_t s) {
    const size_t smem = sizeof(TrainSmem);
    static bool attr[SMEM_MAX_DEVICES] = {};
    cudaError_t e = set_smem_once(mlp_grad_kernel, smem, attr);
    if (e != cudaSuccess) return e;
    return launch_pdl(mlp_grad_kernel, 1, 256, smem, s, m);
}

cudaError_t launch_adam(const MlpArgs &m, float lr, float beta1, float beta2, float eps, float c1, float c2,
                        cudaStream_t s) {
    return launch_pdl(adam_kernel, (NPAR + 255) / 256, 256, 0, s, m, lr, beta1, beta2, eps, c1, c2);
}

cudaError_t launch_to_half(const float *src, __half *dst, int n, cudaStream_t s) {
    to_half_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace lbm

// ---------------------------------------------------------------------------
// trainer (C interface)
// ---------------------------------------------------------------------------

struct lbm_mlp {
    cudaStream_t stream = nullptr;
    __half *par16 = nullptr;
    float *par32 = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr, *loss = nullptr;
    long long t = 0;
};

namespace {

lbm_status mlp_cuda(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

lbm::MlpArgs mlp_args(lbm_mlp *m, const float *x, const float *y, float *out, int n) {
    lbm::MlpArgs a{};
    a.par16 = m->par16;
    a.par32 = m->par32;
    a.adam_m = m->adam_m;
    a.adam_v = m->adam_v;
    a.grad = m->grad;
    a.x = x;
    a.y = y;
    a.out = out;
    a.loss = m->loss;
    a.n = n;
    return a;
}

}  // namespace

extern "C" {

lbm_status lbm_mlp_create(const float *params, void *cuda_stream, lbm_mlp **out) {
    if (!params || !out) return LBM_ERR_ARG;
    *out = nullptr;
    lbm_mlp *m = new lbm_mlp();
    m->stream = (cudaStream_t)cuda_stream;
    const size_t n = lbm::CL_PARAMS;
    bool ok = cudaMalloc(&m->par16, n * sizeof(__half)) == cudaSuccess &&
              cudaMalloc(&m->par32, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->adam_m, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->adam_v, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->grad, n * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->loss, sizeof(float)) == cudaSuccess;
    if (!ok) {
        lbm_mlp_destroy(m);
        return LBM_ERR_OOM;
    }
    ok = cudaMemcpyAsync(m->par32, params, n * sizeof(float), cudaMemcpyHostToDevice, m->stream) == cudaSuccess &&
         cudaMemsetAsync(m->adam_m, 0, n * sizeof(float), m->stream) == cudaSuccess &&
         cudaMemsetAsync(m->adam_v, 0, n * sizeof(float), m->stream) == cudaSuccess &&
         lbm::launch_to_half(m->par32, m->par16, (int)n, m->stream) == cudaSuccess &&
         cudaStreamSynchronize(m->stream) == cudaSuccess;
    if (!ok) {
        lbm_mlp_destroy(m);
        return LBM_ERR_CUDA;
    }
    *out = m;
    return LBM_OK;
}

lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x, float *y, int n) {
    if (!m || n < 0 || (n > 0 && (!x || !y))) return LBM_ERR_ARG;
    return mlp_cuda(lbm::launch_mlp_infer(mlp_args(m, x, nullptr, y, n), nullptr, m->stream));
}

lbm_status lbm_mlp_grad(lbm_mlp *m, const float *x, const float *y, int n, float *grad, float *loss) {
    if (!m || n <= 0 || !x || !y) return LBM_ERR_ARG;
    lbm_status s = mlp_cuda(lbm::launch_mlp_grad(mlp_args(m, x, y, nullptr, n), m->stream));
    if (s != LBM_OK) return s;
    if (grad)
        s = mlp_cuda(cudaMemcpyAsync(grad, m->grad, lbm::CL_PARAMS * sizeof(float), cudaMemcpyDeviceToDevice,
                                     m->stream));
    if (s == LBM_OK && loss) {
        s = mlp_cuda(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        if (s == LBM_OK) s = mlp_cuda(cudaStreamSynchronize(m->stream));
    }
    return s;
}

lbm_status lbm_mlp_train_step(lbm_mlp *m, const float *x, const float *y, int n, float lr, float *loss) {
    if (!m || n <= 0 || !x || !y || !(lr > 0.f)) return LBM_ERR_ARG;
    const lbm::MlpArgs a = mlp_args(m, x, y, nullptr, n);
    lbm_status s = mlp_cuda(lbm::launch_mlp_grad(a, m->stream));
    if (s != LBM_OK) return s;
    m->t += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)m->t)), c2 = (float)(1.0 - std::pow(b2, (double)m->t));
    s = mlp_cuda(lbm::launch_adam(a, lr, (float)b1, (float)b2, 1e-8f, c1, c2, m->stream));
    if (s == LBM_OK && loss) {
        s = mlp_cuda(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        if (s == LBM_OK) s = mlp_cuda(cudaStreamSynchronize(m->stream));
    }
    return s;
}

lbm_status lbm_mlp_get_params(lbm_mlp *m, float *params, void *params_fp16) {
    if (!m) return LBM_ERR_ARG;
    const size_t n = lbm::CL_PARAMS;
    lbm_status s = LBM_OK;
    if (params)
        s = mlp_cuda(cudaMemcpyAsync(params, m->par32, n * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (s == LBM_OK && params_fp16)
        s = mlp_cuda(cudaMemcpyAsync(params_fp16, m->par16, n * sizeof(__half), cudaMemcpyDeviceToHost, m->stream));
    if (s == LBM_OK) s = mlp_cuda(cudaStreamSynchronize(m->stream));
    return s;
}

lbm_status lbm_mlp_destroy(lbm_mlp *m) {
    if (!m) return LBM_ERR_ARG;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    cudaFree(m->par16);
    cudaFree(m->par32);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->grad);
    cudaFree(m->loss);
    delete m;
    return LBM_OK;
}

}  // extern "C"
