// lbm_sbf.cu -- the slender-body formulation (Sec. 3) of rigid straight fibres
// in unbounded Stokes flow, FP64 on the GPU.
//
// Fibre m: centre x_m, unit tangent p_m, half length l_m, radius r_m,
// d_m = -ln((r_m / (2 l_m))^2 e) (Eq. SBFGeomParam).  The line force per unit
// length is F_m / (2 l_m) + sum_{n=1..N} b_m^n P_n(sigma), sigma = s / l_m
// (Eq. force_exp).  Projecting Eq. sev_fils on the Legendre polynomials, with
// Kbar[P_n] = lambda_n P_n, lambda_n = -2 sum_{i<=n} 1/i, and the torque
// condition of Eq. extra_cond (which fixes b^1 across the fibre:
// 3 / (2 l^2) M x p) leaves per fibre the unknowns beta (b^1 along p) and
// b^2..b^N:
//   (4/3)(d + lambda_1) beta_m + p_m . Q_m^1 = 0,
//   (2 / (2n + 1)) A_n b_m^n + Q_m^n = 0   (n >= 2),
// with A_n = Lam + lambda_n (I + p p^T), Lam = d (I + p p^T) + 2 (I - p p^T),
// and the interaction projections Q_m^j = sum_{k != m} sum_n Theta_mk^{jn} b_k^n,
//   Theta_mk^{jn} = int int G(x_m + l_m sigma p_m - x_k - l_k sigma' p_k)
//                   P_j(sigma) P_n(sigma') l_k dsigma' dsigma,
// G = S + r_k^2 / 2 D (Eq. Gnonper), integrated by tensor Gauss-Legendre
// quadrature.  Then (Eqs. xadot, padot)
//   xdot_m = Lam F / (16 pi mu l) + Q_m^0 / (16 pi mu),
//   pdot_m = 3 d (M x p) / (16 pi mu l^3) + 3 / (16 pi mu l) (I - p p^T) Q_m^1.
//
// Kernels: one block per fibre pair for Theta (its inner sum in registers,
// the outer sum through shared memory), one thread per matrix entry for the
// dense system, a single-block Gauss-Jordan elimination with partial
// pivoting (systems of a few hundred unknowns), one warp per fibre for the
// velocities.
#include "lbm_internal.cuh"
#include "lbm_sbf.h"

#include <cmath>
#include <vector>

namespace lbm {
namespace {

constexpr int SBF_MAX_MODES = 10;
constexpr int SBF_MAX_QUAD = 64;
constexpr int SBF_MAX_FIBRES = 64;
constexpr int SBF_THREADS = 64;  // >= SBF_MAX_QUAD

struct SbfDev {
    int M, N, nq, nu;  // fibres, modes, quadrature nodes, unknowns per fibre (1 + 3 (N - 1))
    double mu;
    const double *x, *p, *l, *r, *d;  // per fibre (x, p: 3 each)
    const double *sig, *w, *P;        // nodes, weights, P[n * nq + a] = P_n(sigma_a)
    double *theta;                    // (M, M, N+1, N+1, 3, 3)
    double *aug;                      // n x (n + 1), n = M nu
    const double *F, *T;              // external force and torque (3 per fibre)
    double *z;                        // solution (n)
    double *xdot, *pdot;              // 3 per fibre
    int *status;                      // 0 ok, 1 singular
};

__device__ __forceinline__ double lambda_n(int n) {
    double s = 0.0;
    for (int i = 1; i <= n; ++i) s += 1.0 / i;
    return -2.0 * s;
}

__device__ __forceinline__ size_t theta_at(const SbfDev &s, int m, int k, int j, int n) {
    return ((((size_t)m * s.M + k) * (s.N + 1) + j) * (s.N + 1) + n) * 9;
}

// Theta_mk for every (j, n): block (m, k); thread a handles node sigma_a of
// fibre m and sums over the nodes of fibre k; the sums over a go through
// shared memory.
__global__ void __launch_bounds__(SBF_THREADS) sbf_theta_kernel(SbfDev s) {
    const int m = blockIdx.x / s.M, k = blockIdx.x % s.M;
    const int N1 = s.N + 1;
    __shared__ double H[SBF_MAX_QUAD][SBF_MAX_MODES + 1][6];
    const int a = threadIdx.x;
    if (m == k) {
        for (int e = threadIdx.x; e < N1 * N1 * 9; e += blockDim.x) s.theta[theta_at(s, m, k, 0, 0) + e] = 0.0;
        return;
    }
    if (a < s.nq) {
        double acc[SBF_MAX_MODES + 1][6];
        for (int n = 0; n < N1; ++n)
            for (int c = 0; c < 6; ++c) acc[n][c] = 0.0;
        const double lm = s.l[m], lk = s.l[k], rk = s.r[k];
        double xa[3];
        for (int c = 0; c < 3; ++c) xa[c] = s.x[3 * m + c] + lm * s.sig[a] * s.p[3 * m + c];
        for (int b = 0; b < s.nq; ++b) {
            double R[3];
            for (int c = 0; c < 3; ++c) R[c] = xa[c] - (s.x[3 * k + c] + lk * s.sig[b] * s.p[3 * k + c]);
            const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
            const double ir = 1.0 / sqrt(r2), ir3 = ir / r2;
            const double h = 0.5 * rk * rk;
            // symmetric G: S = (I + R R^T / r^2) / r, D = (I - 3 R R^T / r^2) / r^3
            double g[6];
            const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
            for (int c = 0; c < 6; ++c) {
                const double rr = R[ii[c]] * R[jj[c]] / r2;
                const double del = ii[c] == jj[c] ? 1.0 : 0.0;
                g[c] = (del + rr) * ir + h * (del - 3.0 * rr) * ir3;
            }
            const double wb = s.w[b] * lk;
            for (int n = 0; n < N1; ++n) {
                const double f = wb * s.P[n * s.nq + b];
                for (int c = 0; c < 6; ++c) acc[n][c] += f * g[c];
            }
        }
        const double wa = s.w[a];
        for (int n = 0; n < N1; ++n)
            for (int c = 0; c < 6; ++c) H[a][n][c] = wa * acc[n][c];
    }
    __syncthreads();
    // Theta[j][n][c] = sum_a P_j(sigma_a) H[a][n][c]
    for (int e = threadIdx.x; e < N1 * N1 * 6; e += blockDim.x) {
        const int c = e % 6, jn = e / 6, n = jn % N1, j = jn / N1;
        double t = 0.0;
        for (int aa = 0; aa < s.nq; ++aa) t += s.P[j * s.nq + aa] * H[aa][n][c];
        const size_t o = theta_at(s, m, k, j, n);
        const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
        s.theta[o + 3 * ii[c] + jj[c]] = t;
        s.theta[o + 3 * jj[c] + ii[c]] = t;
    }
}

// Known part of b_k^n (n = 0: F / (2 l); n = 1: 3 / (2 l^2) M x p; else 0).
__device__ __forceinline__ double b_known(const SbfDev &s, int k, int n, int c) {
    if (n == 0) return s.F[3 * k + c] / (2.0 * s.l[k]);
    if (n == 1) {
        const double *M = s.T + 3 * k, *p = s.p + 3 * k;
        const double cr[3] = {M[1] * p[2] - M[2] * p[1], M[2] * p[0] - M[0] * p[2], M[0] * p[1] - M[1] * p[0]};
        return 3.0 / (2.0 * s.l[k] * s.l[k]) * cr[c];
    }
    return 0.0;
}

// d b_k^n[c] / d z_k[u] (the unknowns of fibre k enter b linearly).
__device__ __forceinline__ double b_coef(const SbfDev &s, int k, int n, int c, int u) {
    if (n == 1) return u == 0 ? s.p[3 * k + c] : 0.0;
    if (n >= 2) return (u == 1 + 3 * (n - 2) + c) ? 1.0 : 0.0;
    return 0.0;
}

// Row (m, e) of the projected equations: e = 0 the beta row, e = 1 + 3 (n - 2) + a the
// component a of mode n >= 2.  Fills the augmented matrix entry (row, col), col = n_tot: rhs.
__global__ void sbf_assemble_kernel(SbfDev s) {
    const int n_tot = s.M * s.nu;
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)n_tot * (n_tot + 1)) return;
    const int row = (int)(id / (n_tot + 1)), col = (int)(id % (n_tot + 1));
    const int m = row / s.nu, e = row % s.nu;
    const int N1 = s.N + 1;
    // the row as a linear form on the Q projections: weights v over (j, component)
    // row e = 0: j = 1, weights p_m; row e > 0: j = n, unit vector a
    const int j = e == 0 ? 1 : 2 + (e - 1) / 3;
    const int acomp = e == 0 ? -1 : (e - 1) % 3;
    auto vw = [&](int c) { return acomp < 0 ? s.p[3 * m + c] : (c == acomp ? 1.0 : 0.0); };
    double val = 0.0;
    if (col < n_tot) {
        const int k = col / s.nu, u = col % s.nu;
        if (k != m) {
            // sum_n sum_{a,c} v_a Theta_mk[j][n][a][c] db_k^n[c]/dz_k[u]
            for (int n = 1; n < N1; ++n)
                for (int c = 0; c < 3; ++c) {
                    const double db = b_coef(s, k, n, c, u);
                    if (db == 0.0) continue;
                    const size_t o = theta_at(s, m, k, j, n);
                    for (int aa = 0; aa < 3; ++aa) val += vw(aa) * s.theta[o + 3 * aa + c] * db;
                }
        } else {
            // own terms: (4/3)(d + lambda_1) beta, or (2/(2n+1)) A_n b^n
            const double dm = s.d[m];
            if (e == 0) {
                if (u == 0) val = (4.0 / 3.0) * (dm + lambda_n(1));
            } else {
                const int n = j;
                if (u >= 1 && (u - 1) / 3 == n - 2) {
                    const int c = (u - 1) % 3;
                    const double *p = s.p + 3 * m;
                    const double del = acomp == c ? 1.0 : 0.0, pp = p[acomp] * p[c];
                    const double Lam = dm * (del + pp) + 2.0 * (del - pp);
                    val = 2.0 / (2 * n + 1) * (Lam + lambda_n(n) * (del + pp));
                }
            }
        }
    } else {
        // rhs: -sum_k sum_n v . Theta_mk[j][n] b_known_k^n
        for (int k = 0; k < s.M; ++k) {
            if (k == m) continue;
            for (int n = 0; n < 2; ++n) {
                const size_t o = theta_at(s, m, k, j, n);
                for (int aa = 0; aa < 3; ++aa)
                    for (int c = 0; c < 3; ++c) val -= vw(aa) * s.theta[o + 3 * aa + c] * b_known(s, k, n, c);
            }
        }
    }
    s.aug[(size_t)row * (n_tot + 1) + col] = val;
}

// Gauss-Jordan elimination with partial pivoting on the augmented matrix, one block.
__global__ void __launch_bounds__(256) sbf_solve_kernel(SbfDev s) {
    const int n = s.M * s.nu, w = n + 1;
    double *A = s.aug;
    __shared__ double best[256];
    __shared__ int bidx[256];
    __shared__ int piv;
    for (int col = 0; col < n; ++col) {
        double bv = -1.0;
        int bi = col;
        for (int i = col + threadIdx.x; i < n; i += blockDim.x) {
            const double v = fabs(A[(size_t)i * w + col]);
            if (v > bv) { bv = v; bi = i; }
        }
        best[threadIdx.x] = bv;
        bidx[threadIdx.x] = bi;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -1.0;
            int bi0 = col;
            for (int t = 0; t < (int)blockDim.x; ++t)
                if (best[t] > b) { b = best[t]; bi0 = bidx[t]; }
            piv = bi0;
            if (!(b > 1e-300)) *s.status = 1;
        }
        __syncthreads();
        const int pr = piv;
        if (pr != col)
            for (int c = threadIdx.x; c < w; c += blockDim.x) {
                const double t = A[(size_t)col * w + c];
                A[(size_t)col * w + c] = A[(size_t)pr * w + c];
                A[(size_t)pr * w + c] = t;
            }
        __syncthreads();
        const double inv = 1.0 / A[(size_t)col * w + col];
        __syncthreads();
        for (int c = threadIdx.x; c < w; c += blockDim.x) A[(size_t)col * w + c] *= inv;
        __syncthreads();
        for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
            const int i = e / w, c = e % w;
            if (i == col || c == col) continue;
            A[(size_t)i * w + c] -= A[(size_t)i * w + col] * A[(size_t)col * w + c];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            if (i != col) A[(size_t)i * w + col] = 0.0;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) s.z[i] = A[(size_t)i * w + n];
}

// Velocities of fibre m (one warp; lane 0 writes).
__global__ void sbf_velocity_kernel(SbfDev s) {
    const int m = blockIdx.x;
    if (threadIdx.x != 0) return;
    const int N1 = s.N + 1;
    double Q0[3] = {0, 0, 0}, Q1[3] = {0, 0, 0};
    for (int k = 0; k < s.M; ++k) {
        if (k == m) continue;
        for (int n = 0; n < N1; ++n) {
            double b[3];
            for (int c = 0; c < 3; ++c) {
                b[c] = b_known(s, k, n, c);
                for (int u = 0; u < s.nu; ++u) b[c] += b_coef(s, k, n, c, u) * s.z[k * s.nu + u];
            }
            const size_t o0 = theta_at(s, m, k, 0, n), o1 = theta_at(s, m, k, 1, n);
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) {
                    Q0[a] += s.theta[o0 + 3 * a + c] * b[c];
                    Q1[a] += s.theta[o1 + 3 * a + c] * b[c];
                }
        }
    }
    const double *p = s.p + 3 * m, *F = s.F + 3 * m, *M = s.T + 3 * m;
    const double dm = s.d[m], lm = s.l[m], mu = s.mu;
    const double pF = p[0] * F[0] + p[1] * F[1] + p[2] * F[2];
    const double pQ = p[0] * Q1[0] + p[1] * Q1[1] + p[2] * Q1[2];
    const double MxP[3] = {M[1] * p[2] - M[2] * p[1], M[2] * p[0] - M[0] * p[2], M[0] * p[1] - M[1] * p[0]};
    const double pi = 3.14159265358979323846;
    for (int a = 0; a < 3; ++a) {
        // Lam F = d (F + p (p.F)) + 2 (F - p (p.F))
        const double LF = dm * (F[a] + p[a] * pF) + 2.0 * (F[a] - p[a] * pF);
        s.xdot[3 * m + a] = LF / (16.0 * pi * mu * lm) + Q0[a] / (16.0 * pi * mu);
        s.pdot[3 * m + a] = 3.0 * dm * MxP[a] / (16.0 * pi * mu * lm * lm * lm) +
                            3.0 / (16.0 * pi * mu * lm) * (Q1[a] - p[a] * pQ);
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's iteration on P_n
// from Chebyshev initial guesses (Golub-Welsch not needed at these orders).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_sbf {
    int M = 0, N = 0, nq = 0;
    double mu = 0.0;
    cudaStream_t stream = nullptr;
    double *buf = nullptr;  // one device allocation for everything
    size_t buf_doubles = 0;
    int *status = nullptr;
    bool has_fibres = false;
};

extern "C" {

lbm_status lbm_sbf_create(int nfibres, int n_modes, int n_quad, double mu, void *cuda_stream, lbm_sbf **out) {
    if (!out || nfibres < 1 || nfibres > SBF_MAX_FIBRES || n_modes < 2 || n_modes > SBF_MAX_MODES || n_quad < 2 ||
        n_quad > SBF_MAX_QUAD || !(mu > 0.0))
        return LBM_ERR_ARG;
    lbm_sbf *s = new lbm_sbf();
    s->M = nfibres;
    s->N = n_modes;
    s->nq = n_quad;
    s->mu = mu;
    s->stream = (cudaStream_t)cuda_stream;
    const size_t M = nfibres, N1 = n_modes + 1, nq = n_quad, nu = 1 + 3 * (n_modes - 1), n = M * nu;
    s->buf_doubles = 3 * M + 3 * M + M + M + M + nq + nq + N1 * nq + M * M * N1 * N1 * 9 + n * (n + 1) + 3 * M +
                     3 * M + n + 3 * M + 3 * M;
    if (cudaMalloc(&s->buf, sizeof(double) * s->buf_doubles) != cudaSuccess ||
        cudaMalloc(&s->status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (s->buf) cudaFree(s->buf);
        delete s;
        return LBM_ERR_OOM;
    }
    *out = s;
    return LBM_OK;
}

namespace {
SbfDev sbf_view(lbm_sbf *s) {
    SbfDev d;
    const size_t M = s->M, N1 = s->N + 1, nq = s->nq;
    d.M = s->M;
    d.N = s->N;
    d.nq = s->nq;
    d.nu = 1 + 3 * (s->N - 1);
    d.mu = s->mu;
    const size_t n = M * d.nu;
    double *q = s->buf;
    d.x = q; q += 3 * M;
    d.p = q; q += 3 * M;
    d.l = q; q += M;
    d.r = q; q += M;
    d.d = q; q += M;
    d.sig = q; q += nq;
    d.w = q; q += nq;
    d.P = q; q += N1 * nq;
    d.theta = q; q += M * M * N1 * N1 * 9;
    d.aug = q; q += n * (n + 1);
    d.F = q; q += 3 * M;
    d.T = q; q += 3 * M;
    d.z = q; q += n;
    d.xdot = q; q += 3 * M;
    d.pdot = q; q += 3 * M;
    d.status = s->status;
    return d;
}
}  // namespace

lbm_status lbm_sbf_set_fibres(lbm_sbf *s, const double *centres, const double *tangents, const double *half_lengths,
                              const double *radii) {
    if (!s || !centres || !tangents || !half_lengths || !radii) return LBM_ERR_ARG;
    const int M = s->M, N = s->N, nq = s->nq;
    std::vector<double> host(3 * M + 3 * M + M + M + M + nq + nq + (N + 1) * nq);
    double *x = host.data(), *p = x + 3 * M, *l = p + 3 * M, *r = l + M, *d = r + M, *sig = d + M, *w = sig + nq,
           *P = w + nq;
    for (int m = 0; m < M; ++m) {
        const double nrm = std::sqrt(tangents[3 * m] * tangents[3 * m] + tangents[3 * m + 1] * tangents[3 * m + 1] +
                                     tangents[3 * m + 2] * tangents[3 * m + 2]);
        if (!(nrm > 0.0) || !(half_lengths[m] > 0.0) || !(radii[m] > 0.0) || radii[m] >= half_lengths[m])
            return LBM_ERR_ARG;
        for (int c = 0; c < 3; ++c) {
            x[3 * m + c] = centres[3 * m + c];
            p[3 * m + c] = tangents[3 * m + c] / nrm;
        }
        l[m] = half_lengths[m];
        r[m] = radii[m];
        const double eps = radii[m] / (2.0 * half_lengths[m]);
        d[m] = -std::log(eps * eps * std::exp(1.0));
        // every mode's local operator must be invertible: d + lambda_n != 0 and != -2
        double lam = 0.0;
        for (int n = 1; n <= N; ++n) {
            lam -= 2.0 / n;
            if (std::fabs(d[m] + lam) < 1e-6 || std::fabs(d[m] + lam + 2.0) < 1e-6) return LBM_ERR_ARG;
        }
    }
    std::vector<double> gx, gw;
    gauss_legendre(nq, gx, gw);
    for (int a = 0; a < nq; ++a) {
        sig[a] = gx[a];
        w[a] = gw[a];
        double p0 = 1.0, p1 = gx[a];
        P[a] = 1.0;
        if (N >= 1) P[nq + a] = gx[a];
        for (int n = 2; n <= N; ++n) {
            const double p2 = ((2.0 * n - 1.0) * gx[a] * p1 - (n - 1.0) * p0) / n;
            P[n * nq + a] = p2;
            p0 = p1;
            p1 = p2;
        }
    }
    if (cudaMemcpyAsync(s->buf, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, s->stream) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    SbfDev dv = sbf_view(s);
    sbf_theta_kernel<<<M * M, SBF_THREADS, 0, s->stream>>>(dv);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    s->has_fibres = true;
    return LBM_OK;
}

lbm_status lbm_sbf_solve(lbm_sbf *s, const double *force3m, const double *torque3m, double *xdot3m, double *pdot3m) {
    if (!s || !force3m || !torque3m || !xdot3m || !pdot3m) return LBM_ERR_ARG;
    if (!s->has_fibres) return LBM_ERR_STATE;
    SbfDev dv = sbf_view(s);
    const int M = s->M;
    const size_t n = (size_t)M * dv.nu;
    std::vector<double> ft(6 * M);
    for (int i = 0; i < 3 * M; ++i) {
        ft[i] = force3m[i];
        ft[3 * M + i] = torque3m[i];
    }
    if (cudaMemcpyAsync((void *)dv.F, ft.data(), sizeof(double) * 6 * M, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(s->status, 0, sizeof(int), s->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    const long long entries = (long long)n * (n + 1);
    sbf_assemble_kernel<<<(unsigned)((entries + 255) / 256), 256, 0, s->stream>>>(dv);
    sbf_solve_kernel<<<1, 256, 0, s->stream>>>(dv);
    sbf_velocity_kernel<<<M, 32, 0, s->stream>>>(dv);
    if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
    std::vector<double> v(6 * M);
    int st = 0;
    if (cudaMemcpyAsync(v.data(), dv.xdot, sizeof(double) * 6 * M, cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (st) return LBM_ERR_NUMERIC;
    for (int i = 0; i < 3 * M; ++i) {
        xdot3m[i] = v[i];
        pdot3m[i] = v[3 * M + i];
    }
    return LBM_OK;
}

lbm_status lbm_sbf_destroy(lbm_sbf *s) {
    if (!s) return LBM_ERR_ARG;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->buf);
    cudaFree(s->status);
    delete s;
    return LBM_OK;
}

}  // extern "C"
