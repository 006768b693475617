// Self-consistent screening of the atomic polarisabilities (the MBD@rsSCS
// front end).  arXiv 2307.02278 names this step in its review of the MBD model
// (the polarisabilities, made frequency-dependent, are screened by a Dyson-like
// equation solved at a set of frequencies) and keeps it out of its own scope;
// the published range-separated scheme is restated:
//   alpha_i(iu) = alpha_i / (1 + (u/omega_i)^2),  sigma_i(u) = (sqrt(2/pi) alpha_i(iu) / 3)^(1/3)
//   T_SR_ij(u)  = sum'_n (1 - f(|r+n|)) T_GG(r+n; sqrt(sigma_i^2 + sigma_j^2)),  |r+n| < damp_cut
//   T_GG(r; s)  = grad_i grad_j erf(|r|/s)/|r| = c_id I - c_rr r r^T,  f = the Fermi damping s(R; beta)
//   (A(u)^-1 + T_SR(u)) X_c = 1_c  (c = x, y, z),   alpha_i^SCS(iu) = (1/3) sum_c X_c[i, c]
//   C6_i = (3/pi) int_0^inf alpha_i^SCS(iu)^2 du,  omega_i^SCS = 4 C6_i / (3 alpha_i^SCS(0)^2),
//   Rvdw_i^SCS = Rvdw_i (alpha_i^SCS(0) / alpha_i)^(1/3).
//
// GB300 layout: the columns of the solve are (direction c, frequency k), the
// frequency innermost in 32 lanes (k = 0 static, 1..n the quadrature nodes).
// A warp owns an atom, lane k its frequency, and the three directions share
// the lane's tensor.  Mixed systems evaluate T_SR in FP32 inside every product
// from a 16-byte record per pair {r, (1 - f) [r < damp_cut]} and the squared
// widths sigma_j(u_k)^2 (one coalesced row per neighbour): the product then
// costs arithmetic, not a pass over stored tensors (32 x 6 values per pair).
// FP64 systems evaluate T_SR once per call in FP64 and keep it, [nnz][6][32],
// streamed once per step.  Vectors are FP64 [N][3 a][3 c][32]; the search
// direction also in the operator precision for the neighbour gathers.  Jacobi
// preconditioner diag(alpha_i(iu)).  Column sums are deterministic: fixed
// grid, warps take atoms in a fixed stride, block partials summed in block
// order.
#include "mbd_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mbd {
namespace {

constexpr int kLanes = 32;                  // frequency columns per direction
constexpr int kCols = 3 * kLanes;           // (c, k)
constexpr int kVec = 9 * kLanes;            // values per atom: [a][c][k]
constexpr int kWarps = 8;                   // warps per block
constexpr double kU0 = 0.5;                 // centre of the frequency map (Ha)
constexpr double kPiD = 3.14159265358979323846;

// Gauss-Legendre nodes and weights on (-1, 1) by Newton's method on the
// Legendre polynomial P_n (three-term recurrence), started from the
// asymptotic guesses cos(pi (i - 1/4) / (n + 1/2)); w = 2 / ((1 - t^2) P_n'(t)^2).
void gauss_legendre(int n, std::vector<double> &t, std::vector<double> &w) {
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPiD * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pn = n == 1 ? x : p1, pm = n == 1 ? 1.0 : p0;
            dp = n * (x * pn - pm) / (x * x - 1.0);
            const double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pn = n == 1 ? x : p1, pm = n == 1 ? 1.0 : p0;
        dp = n * (x * pn - pm) / (x * x - 1.0);
        t[n - 1 - i] = x;                    // ascending
        w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

struct ScsArgs {
    int N, ncol;
    const double *alpha, *omega, *rvdw, *pos;
    const int *row, *col, *shift;
    double cell[9];
    double damp_cut, damp_beta, damp_d;
    const double *u;            // [32] frequencies (0 beyond ncol)
};

// Per atom and column: 1 / alpha_i(iu_k), alpha_i(iu_k), sigma_i(u_k) and
// sigma_i(u_k)^2 in FP32; zeros beyond ncol.
__global__ void k_scs_atoms(ScsArgs a, double *__restrict__ ainv, double *__restrict__ aiu, double *__restrict__ sig,
                            float *__restrict__ sig2f) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N * kLanes) return;
    const int i = idx / kLanes, k = idx % kLanes;
    double inv = 0.0, au = 0.0, s = 0.0;
    if (k < a.ncol) {
        const double q = a.u[k] / a.omega[i];
        au = a.alpha[i] / (1.0 + q * q);
        inv = 1.0 / au;
        s = cbrt(sqrt(2.0 / kPiD) * au / 3.0);
    }
    ainv[idx] = inv;
    aiu[idx] = au;
    sig[idx] = s;
    sig2f[idx] = float(s * s);
}

// Pair records of the FP32 product: {r_x, r_y, r_z, (1 - f(r)) [r < damp_cut]},
// r = R_i - R_j - n (FP64 from the positions and the image shift); a warp per
// atom, lanes over its entries.
__global__ void k_scs_geometry(ScsArgs a, float4 *__restrict__ geo) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= a.N) return;
    const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2];
    for (int e = a.row[i] + lane; e < a.row[i + 1]; e += 32) {
        const int j = a.col[e];
        const int sh = a.shift[e];
        const double n1 = double((sh & 255) - 128), n2 = double(((sh >> 8) & 255) - 128),
                     n3 = double(((sh >> 16) & 255) - 128);
        const double rx = xi - a.pos[3 * j] - (n1 * a.cell[0] + n2 * a.cell[3] + n3 * a.cell[6]);
        const double ry = yi - a.pos[3 * j + 1] - (n1 * a.cell[1] + n2 * a.cell[4] + n3 * a.cell[7]);
        const double rz = zi - a.pos[3 * j + 2] - (n1 * a.cell[2] + n2 * a.cell[5] + n3 * a.cell[8]);
        const double r = sqrt(rx * rx + ry * ry + rz * rz);
        double oms = 0.0;
        if (r < a.damp_cut)
            oms = 1.0 / (1.0 + exp(a.damp_d * (r / (a.damp_beta * (a.rvdw[i] + a.rvdw[j])) - 1.0)));
        geo[e] = make_float4(float(rx), float(ry), float(rz), float(oms));
    }
}

// T_SR per (pair entry, frequency): a warp per atom i walks its entries, lane
// k evaluates the frequency-k tensor (FP64) and stores it in T.
template <class T>
__global__ void k_scs_tensors(ScsArgs a, const double *__restrict__ sig, T *__restrict__ tsr, long long cap) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int k = threadIdx.x & 31;
    if (i >= a.N) return;
    const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2];
    const double si = sig[(size_t)i * kLanes + k];
    const int e1 = (int)min((long long)a.row[i + 1], cap);
    for (int e = a.row[i]; e < e1; ++e) {
        const int j = a.col[e];
        const int sh = a.shift[e];
        const double n1 = double((sh & 255) - 128), n2 = double(((sh >> 8) & 255) - 128),
                     n3 = double(((sh >> 16) & 255) - 128);
        const double rx = xi - a.pos[3 * j] - (n1 * a.cell[0] + n2 * a.cell[3] + n3 * a.cell[6]);
        const double ry = yi - a.pos[3 * j + 1] - (n1 * a.cell[1] + n2 * a.cell[4] + n3 * a.cell[7]);
        const double rz = zi - a.pos[3 * j + 2] - (n1 * a.cell[2] + n2 * a.cell[5] + n3 * a.cell[8]);
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double r = sqrt(r2);
        double v[6] = {0, 0, 0, 0, 0, 0};
        if (k < a.ncol && r < a.damp_cut) {
            const double sj = sig[(size_t)j * kLanes + k];
            const double s = sqrt(si * si + sj * sj);
            const double x = r / s;
            const double big_e = erf(x), ex = exp(-x * x);
            const double kk = 2.0 / sqrt(kPiD);
            const double inv_r2 = 1.0 / r2, inv_r = 1.0 / r;
            const double cid = big_e * inv_r2 * inv_r - kk * ex / s * inv_r2;
            const double crr = 3.0 * big_e * inv_r2 * inv_r2 * inv_r - 3.0 * kk * ex / s * inv_r2 * inv_r2 -
                               2.0 * kk * ex / (s * s * s) * inv_r2;
            const double oms = 1.0 / (1.0 + exp(a.damp_d * (r / (a.damp_beta * (a.rvdw[i] + a.rvdw[j])) - 1.0)));
            v[0] = oms * (cid - crr * rx * rx);
            v[1] = -oms * crr * rx * ry;
            v[2] = -oms * crr * rx * rz;
            v[3] = oms * (cid - crr * ry * ry);
            v[4] = -oms * crr * ry * rz;
            v[5] = oms * (cid - crr * rz * rz);
        }
        T *o = tsr + (size_t)e * 6 * kLanes + k;
#pragma unroll
        for (int c = 0; c < 6; ++c) o[c * kLanes] = T(v[c]);
    }
}

// Block partial sums of per-lane column values acc[c] (c = 0..2) over the
// block's warps, in warp order: partial[blockIdx.x][c * 32 + lane].
__device__ __forceinline__ void block_columns(const double acc[3], double *__restrict__ partial) {
    __shared__ double s_acc[kWarps][kCols];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 3; ++c) s_acc[warp][c * kLanes + lane] = acc[c];
    __syncthreads();
    for (int t = threadIdx.x; t < kCols; t += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += s_acc[w][t];
        partial[(size_t)blockIdx.x * kCols + t] = s;
    }
}

// q = (A^-1 + T_SR) p; with PQ, also the block partials of p.q per column.
template <class T, bool PQ>
__global__ void __launch_bounds__(kWarps * 32) k_scs_matvec(int N, const int *__restrict__ row,
                                                            const int *__restrict__ col, const T *__restrict__ tsr,
                                                            const T *__restrict__ pT, const double *__restrict__ p,
                                                            const double *__restrict__ ainv, double *__restrict__ q,
                                                            double *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5), nw = gridDim.x * kWarps;
    double dot[3] = {0.0, 0.0, 0.0};
    for (int i = gw; i < N; i += nw) {
        T acc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = T(0);
        for (int e = row[i]; e < row[i + 1]; ++e) {
            const int j = col[e];
            const T *te = tsr + (size_t)e * 6 * kLanes + lane;
            const T t0 = te[0], t1 = te[kLanes], t2 = te[2 * kLanes], t3 = te[3 * kLanes], t4 = te[4 * kLanes],
                    t5 = te[5 * kLanes];
            const T *pj = pT + (size_t)j * kVec + lane;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T x = pj[(0 * 3 + c) * kLanes], y = pj[(1 * 3 + c) * kLanes], z = pj[(2 * 3 + c) * kLanes];
                acc[0 * 3 + c] += t0 * x + t1 * y + t2 * z;
                acc[1 * 3 + c] += t1 * x + t3 * y + t4 * z;
                acc[2 * 3 + c] += t2 * x + t4 * y + t5 * z;
            }
        }
        const double ai = ainv[(size_t)i * kLanes + lane];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const size_t o = (size_t)i * kVec + t * kLanes + lane;
            const double pv = p[o];
            const double qv = ai * pv + double(acc[t]);
            q[o] = qv;
            if (PQ) dot[t % 3] += pv * qv;
        }
    }
    if (PQ) block_columns(dot, partial);
}

// D(x) = erf(x) - (2/sqrt(pi)) x exp(-x^2), the combination the Gaussian
// dipole tensor needs (c_id = D/r^3), in FP32 from e = exp(-x^2):
//   x < 1: its Maclaurin series (2/sqrt(pi)) sum_{n>=1} (-1)^(n+1) 2n x^(2n+1) / (n! (2n+1)),
//          ten terms (truncation below 6e-8 relative), free of the cancellation
//          of the difference at small x;
//   x >= 1: Hastings' rational approximation of erf (Abramowitz & Stegun 7.1.26,
//          |error| <= 1.5e-7), erf = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e,
//          t = 1 / (1 + 0.3275911 x); D >= 0.43 there (relative error below 2.5e-7).
__device__ __forceinline__ float gauss_dipole_d(const float x, const float e) {
    const float kk = 1.1283791670955126f;   // 2 / sqrt(pi)
    if (x < 1.0f) {
        const float x2 = x * x;
        float sr = -2.624506592760561e-07f;
        sr = sr * x2 + 2.6106934001670845e-06f;
        sr = sr * x2 - 2.334267040149393e-05f;
        sr = sr * x2 + 1.8518518518518518e-04f;
        sr = sr * x2 - 1.282051282051282e-03f;
        sr = sr * x2 + 7.575757575757576e-03f;
        sr = sr * x2 - 3.7037037037037035e-02f;
        sr = sr * x2 + 1.4285714285714285e-01f;
        sr = sr * x2 - 0.4f;
        sr = sr * x2 + 0.6666666666666666f;
        return kk * x * x2 * sr;
    }
    const float t = __frcp_rn(1.0f + 0.3275911f * x);
    const float poly = t * (0.254829592f + t * (-0.284496736f + t * (1.421413741f + t * (-1.453152027f +
                                                                                     t * 1.061405429f))));
    return 1.0f - poly * e - kk * x * e;
}

// acc += T_SR(g; s2) x for one pair record g = {r, 1 - f} and squared width s2
// (nothing when either is zero: a lane beyond the columns, a pair beyond the cutoff).
__device__ __forceinline__ void pair_apply(const float4 g, const float s2, const float x[9], float acc[9]) {
    if (!(s2 > 0.0f && g.w > 0.0f)) return;
    const float kk = 1.1283791670955126f;   // 2 / sqrt(pi)
    const float r2 = g.x * g.x + g.y * g.y + g.z * g.z;
    const float inv_r = rsqrtf(r2), inv_s = rsqrtf(s2);
    const float inv_r2 = inv_r * inv_r;
    const float xr = r2 * inv_r * inv_s;
    const float e = expf(-xr * xr);
    const float ke = kk * e * inv_s;
    const float base = gauss_dipole_d(xr, e) * inv_r * inv_r2;
    const float cid = g.w * base;
    const float crr = g.w * (3.0f * base - 2.0f * ke * inv_s * inv_s) * inv_r2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float px = x[0 * 3 + c], py = x[1 * 3 + c], pz = x[2 * 3 + c];
        const float rd = crr * (g.x * px + g.y * py + g.z * pz);
        acc[0 * 3 + c] += cid * px - g.x * rd;
        acc[1 * 3 + c] += cid * py - g.y * rd;
        acc[2 * 3 + c] += cid * pz - g.z * rd;
    }
}

// The same product with T_SR evaluated in FP32 per (pair, frequency):
//   s^2 = sigma_i^2 + sigma_j^2, x = r/s, ke = (2/sqrt(pi)) exp(-x^2)/s,
//   c_id = (1 - f) D(x)/r^3,  c_rr = (1 - f) (3 D(x)/r^3 - 2 ke/s^2)/r^2,
//   T_SR p = c_id p - c_rr r (r . p).
template <bool PQ>
__global__ void __launch_bounds__(kWarps * 32) k_scs_matvec_fly(int N, const int *__restrict__ order,
                                                                const int *__restrict__ row,
                                                                const int *__restrict__ col,
                                                                const float4 *__restrict__ geo,
                                                                const float *__restrict__ sig2,
                                                                const float *__restrict__ pT,
                                                                const double *__restrict__ p,
                                                                const double *__restrict__ ainv,
                                                                double *__restrict__ q,
                                                                double *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5), nw = gridDim.x * kWarps;
    double dot[3] = {0.0, 0.0, 0.0};
    for (int w = gw; w < N; w += nw) {
        const int i = order[w];
        float acc[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[t] = 0.0f;
        const float si2 = sig2[(size_t)i * kLanes + lane];
        // two pair entries per iteration: independent load chains
        const int e0 = row[i], e1 = row[i + 1];
        for (int e = e0; e < e1; e += 2) {
            const bool two = e + 1 < e1;
            const int ja = col[e], jb = two ? col[e + 1] : ja;
            const float4 ga = geo[e], gb = two ? geo[e + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float sa = sig2[(size_t)ja * kLanes + lane], sb = sig2[(size_t)jb * kLanes + lane];
            const float *pa = pT + (size_t)ja * kVec + lane, *pb = pT + (size_t)jb * kVec + lane;
            float xa[9], xb[9];
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                xa[t] = pa[t * kLanes];
                xb[t] = pb[t * kLanes];
            }
            pair_apply(ga, si2 + sa, xa, acc);
            pair_apply(gb, si2 + sb, xb, acc);
        }
        const double ai = ainv[(size_t)i * kLanes + lane];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const size_t o = (size_t)i * kVec + t * kLanes + lane;
            const double pv = p[o];
            const double qv = ai * pv + double(acc[t]);
            q[o] = qv;
            if (PQ) dot[t % 3] += pv * qv;
        }
    }
    if (PQ) block_columns(dot, partial);
}

// Column sums of the block partials: a warp per column, lane l adds the
// blocks l, l + 32, ... in order, then a fixed shuffle tree.
__global__ void k_scs_sum(const double *__restrict__ partial, int nblk, int nsum, double *__restrict__ out) {
    const int t = blockIdx.x;                  // column of the nsum x 96 outputs
    const int lane = threadIdx.x;
    if (t >= nsum * kCols) return;
    const int which = t / kCols, colx = t % kCols;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += partial[((size_t)which * nblk + b) * kCols + colx];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[t] = s;
}

// CG scalars per column.  st[0..95] rho = r.z, st[96..191] alpha step,
// st[192..287] beta, st[288..383] r.r; flags[0] set when p.q <= 0 on a live column.
__global__ void k_scs_alpha(const double *__restrict__ pq, double *__restrict__ st, int *__restrict__ flags) {
    const int t = threadIdx.x;
    if (t >= kCols) return;
    const double rho = st[t], g = pq[t];
    double al = 0.0;
    if (rho > 0.0) {
        if (g > 0.0) al = rho / g;
        else atomicOr(flags, 1);
    }
    st[kCols + t] = al;
}
__global__ void k_scs_beta(const double *__restrict__ sums, double *__restrict__ st, int first) {
    const int t = threadIdx.x;
    if (t >= kCols) return;
    const double rho_new = sums[t], rho_old = st[t];
    st[2 * kCols + t] = (first || rho_old <= 0.0) ? 0.0 : rho_new / rho_old;
    st[t] = rho_new;
    st[3 * kCols + t] = sums[kCols + t];
}

// x += a p, r -= a q (first: x = x0 = p, r = b - q), with the block partials of
// r.z (z = alpha_i(iu) r) and r.r per column.
__global__ void __launch_bounds__(kWarps * 32) k_scs_update(int N, int first, const double *__restrict__ st,
                                                            const double *__restrict__ p,
                                                            const double *__restrict__ q,
                                                            const double *__restrict__ aiu, double *__restrict__ x,
                                                            double *__restrict__ r, double *__restrict__ partial,
                                                            int nblk) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5), nw = gridDim.x * kWarps;
    double rz[3] = {0.0, 0.0, 0.0}, rr[3] = {0.0, 0.0, 0.0};
    double al[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) al[c] = first ? 0.0 : st[kCols + c * kLanes + lane];
    for (int i = gw; i < N; i += nw) {
        const double zscale = aiu[(size_t)i * kLanes + lane];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int a = t / 3, c = t % 3;
            const size_t o = (size_t)i * kVec + t * kLanes + lane;
            double rv;
            if (first) {
                x[o] = p[o];
                rv = (a == c && zscale > 0.0 ? 1.0 : 0.0) - q[o];
            } else {
                x[o] += al[c] * p[o];
                rv = r[o] - al[c] * q[o];
            }
            r[o] = rv;
            rz[c] += rv * (rv * zscale);
            rr[c] += rv * rv;
        }
    }
    block_columns(rz, partial);
    __syncthreads();
    block_columns(rr, partial + (size_t)nblk * kCols);
}

// p = z + beta p (first: p = x0 = alpha_i(iu) delta_ac), and its copy in T.
template <class T>
__global__ void k_scs_direction(int N, int mode, const double *__restrict__ st, const double *__restrict__ r,
                                const double *__restrict__ aiu, double *__restrict__ p, T *__restrict__ pT) {
    const size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= (size_t)N * kVec) return;
    const int lane = (int)(o % kLanes), t = (int)((o / kLanes) % 9), i = (int)(o / kVec);
    const int a = t / 3, c = t % 3;
    const double zs = aiu[(size_t)i * kLanes + lane];
    double v;
    if (mode == 0) v = (a == c) ? zs : 0.0;                                       // x0 = A 1_c
    else v = r[o] * zs + st[2 * kCols + c * kLanes + lane] * p[o];
    p[o] = v;
    pT[o] = T(v);
}

// Screened outputs per atom from the solutions x.
__global__ void k_scs_finish(int N, int ncol, const double *__restrict__ x, const double *__restrict__ alpha,
                             const double *__restrict__ rvdw, const double *__restrict__ wq,
                             double *__restrict__ out, double *__restrict__ aiu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double a0 = 0.0, c6 = 0.0;
    for (int k = 0; k < ncol; ++k) {
        const size_t b = (size_t)i * kVec + k;
        const double ak = (x[b + 0 * kLanes] + x[b + 4 * kLanes] + x[b + 8 * kLanes]) / 3.0;
        aiu[(size_t)k * N + i] = ak;
        if (k == 0) a0 = ak;
        else c6 += wq[k] * ak * ak;
    }
    c6 *= 3.0 / kPiD;
    out[i] = a0;
    out[N + i] = 4.0 * c6 / (3.0 * a0 * a0);
    out[2 * N + i] = rvdw[i] * cbrt(a0 / alpha[i]);
    out[3 * N + i] = c6;
}

template <class T>
mbd_status screen(mbd_system *s, int n_freq, double tol, int max_iter, double *alpha_out, double *omega_out,
                  double *rvdw_out, double *c6_out, double *aiu_out, int32_t *iters_out, double *res_out) {
    const int N = s->N, ncol = n_freq + 1;
    const cudaStream_t st = s->stream;
    std::vector<double> t, w;
    gauss_legendre(n_freq, t, w);
    std::vector<double> u(kLanes, 0.0), wq(kLanes, 0.0);
    for (int k = 0; k < n_freq; ++k) {
        u[k + 1] = kU0 * (1.0 + t[k]) / (1.0 - t[k]);
        wq[k + 1] = w[k] * 2.0 * kU0 / ((1.0 - t[k]) * (1.0 - t[k]));
    }
    const long long nnz = s->nnz;
    constexpr bool kFly = sizeof(T) == 4;   // FP32 operator: T_SR evaluated inside each product
    DevBuf d_u, d_wq, d_al, d_om, d_ainv, d_aiu_c, d_sig, d_sig2, d_geo, d_tsr, d_x, d_r, d_p, d_q, d_pT, d_part, d_sums, d_st,
        d_flag,
        d_out, d_aiu;
    const size_t nv = (size_t)N * kVec;
    // persistent grid: the resident blocks of the product kernel on every SM
    int per_sm = 0;
    if constexpr (kFly)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scs_matvec_fly<true>, kWarps * 32, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scs_matvec<T, true>, kWarps * 32, 0);
    cudaGetLastError();
    per_sm = std::max(1, std::min(8, per_sm));
    const int nblk = std::max(1, std::min((N + kWarps - 1) / kWarps, per_sm * std::max(1, s->num_sms)));
    MBD_TRY(d_u.ensure(kLanes * sizeof(double)));
    MBD_TRY(d_wq.ensure(kLanes * sizeof(double)));
    MBD_TRY(d_al.ensure(N * sizeof(double)));
    MBD_TRY(d_om.ensure(N * sizeof(double)));
    MBD_TRY(d_ainv.ensure((size_t)N * kLanes * sizeof(double)));
    MBD_TRY(d_aiu_c.ensure((size_t)N * kLanes * sizeof(double)));
    MBD_TRY(d_sig.ensure((size_t)N * kLanes * sizeof(double)));
    MBD_TRY(d_sig2.ensure((size_t)N * kLanes * sizeof(float)));
    if constexpr (kFly)
        MBD_TRY(d_geo.ensure(std::max<size_t>(1, (size_t)nnz) * sizeof(float4)));
    else
        MBD_TRY(d_tsr.ensure(std::max<size_t>(1, (size_t)nnz) * 6 * kLanes * sizeof(T)));
    MBD_TRY(d_x.ensure(nv * sizeof(double)));
    MBD_TRY(d_r.ensure(nv * sizeof(double)));
    MBD_TRY(d_p.ensure(nv * sizeof(double)));
    MBD_TRY(d_q.ensure(nv * sizeof(double)));
    MBD_TRY(d_pT.ensure(nv * sizeof(T)));
    MBD_TRY(d_part.ensure((size_t)2 * nblk * kCols * sizeof(double)));
    MBD_TRY(d_sums.ensure(2 * kCols * sizeof(double)));
    MBD_TRY(d_st.ensure(4 * kCols * sizeof(double)));
    MBD_TRY(d_flag.ensure(sizeof(int)));
    MBD_TRY(d_out.ensure(4 * (size_t)N * sizeof(double)));
    MBD_TRY(d_aiu.ensure((size_t)ncol * N * sizeof(double)));
    MBD_CUDA_TRY(cudaMemcpyAsync(d_u.ptr, u.data(), kLanes * sizeof(double), cudaMemcpyHostToDevice, st));
    MBD_CUDA_TRY(cudaMemcpyAsync(d_wq.ptr, wq.data(), kLanes * sizeof(double), cudaMemcpyHostToDevice, st));
    MBD_CUDA_TRY(cudaMemcpyAsync(d_al.ptr, s->alpha.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
    MBD_CUDA_TRY(cudaMemcpyAsync(d_om.ptr, s->omega.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
    MBD_CUDA_TRY(cudaMemsetAsync(d_flag.ptr, 0, sizeof(int), st));
    MBD_CUDA_TRY(cudaMemsetAsync(d_st.ptr, 0, 4 * kCols * sizeof(double), st));

    ScsArgs a{};
    a.N = N;
    a.ncol = ncol;
    a.alpha = d_al.as<double>();
    a.omega = d_om.as<double>();
    a.rvdw = s->rvdw_d.as<double>();
    a.pos = s->pos_d.as<double>();
    a.row = s->row_d.as<int>();
    a.col = s->col_d.as<int>();
    a.shift = s->shift_d.as<int>();
    for (int c = 0; c < 9; ++c) a.cell[c] = s->cell[c];
    a.damp_cut = s->damp_cut;
    a.damp_beta = s->damp_beta;
    a.damp_d = s->damp_d;
    a.u = d_u.as<double>();

    k_scs_atoms<<<(N * kLanes + 255) / 256, 256, 0, st>>>(a, d_ainv.as<double>(), d_aiu_c.as<double>(),
                                                          d_sig.as<double>(),
                                                          d_sig2.as<float>());
    MBD_LAUNCH_CHECK();
    if constexpr (kFly)
        k_scs_geometry<<<(N + 7) / 8, 256, 0, st>>>(a, d_geo.as<float4>());
    else
        k_scs_tensors<T><<<(N + 7) / 8, 256, 0, st>>>(a, d_sig.as<double>(), d_tsr.as<T>(), nnz);
    MBD_LAUNCH_CHECK();
    auto matvec = [&](bool pq) {
        if constexpr (kFly) {
            auto kern = pq ? k_scs_matvec_fly<true> : k_scs_matvec_fly<false>;
            kern<<<nblk, kWarps * 32, 0, st>>>(N, s->order_d.as<int>(), a.row, a.col, d_geo.as<float4>(),
                                               d_sig2.as<float>(),
                                               reinterpret_cast<const float *>(d_pT.ptr), d_p.as<double>(),
                                               d_ainv.as<double>(), d_q.as<double>(), d_part.as<double>());
        } else {
            auto kern = pq ? k_scs_matvec<T, true> : k_scs_matvec<T, false>;
            kern<<<nblk, kWarps * 32, 0, st>>>(N, a.row, a.col, d_tsr.as<T>(), d_pT.as<T>(), d_p.as<double>(),
                                               d_ainv.as<double>(), d_q.as<double>(), d_part.as<double>());
        }
    };

    const unsigned vgrid = (unsigned)((nv + 255) / 256);
    double *st_d = d_st.as<double>();
    // x0 = A 1_c, r0 = 1_c - M x0, p0 = z0
    k_scs_direction<T><<<vgrid, 256, 0, st>>>(N, 0, st_d, d_r.as<double>(), d_aiu_c.as<double>(), d_p.as<double>(),
                                              d_pT.as<T>());
    matvec(false);
    k_scs_update<<<nblk, kWarps * 32, 0, st>>>(N, 1, st_d, d_p.as<double>(), d_q.as<double>(), d_aiu_c.as<double>(),
                                               d_x.as<double>(), d_r.as<double>(), d_part.as<double>(), nblk);
    k_scs_sum<<<2 * kCols, 32, 0, st>>>(d_part.as<double>(), nblk, 2, d_sums.as<double>());
    k_scs_beta<<<1, kCols, 0, st>>>(d_sums.as<double>(), st_d, 1);
    k_scs_direction<T><<<vgrid, 256, 0, st>>>(N, 1, st_d, d_r.as<double>(), d_aiu_c.as<double>(), d_p.as<double>(),
                                              d_pT.as<T>());
    MBD_LAUNCH_CHECK();

    // convergence: ||r_c,k|| <= tol ||1_c|| = tol sqrt(N) on every live column
    std::vector<double> hst(4 * kCols);
    int iters = 0;
    double worst = 0.0;
    const double bnorm2 = (double)N;
    auto residual = [&](bool &done) -> mbd_status {
        MBD_CUDA_TRY(cudaMemcpyAsync(hst.data(), st_d, 4 * kCols * sizeof(double), cudaMemcpyDeviceToHost, st));
        MBD_CUDA_TRY(cudaStreamSynchronize(st));
        worst = 0.0;
        bool finite = true;
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < ncol; ++k) {
                const double rr = hst[3 * kCols + c * kLanes + k];
                finite = finite && std::isfinite(rr);
                worst = std::max(worst, std::sqrt(std::max(rr, 0.0) / bnorm2));
            }
        if (!finite) return MBD_ERR_NONFINITE;
        done = worst <= tol;
        return MBD_OK;
    };
    bool done = false;
    MBD_TRY(residual(done));
    while (!done && iters < max_iter) {
        matvec(true);
        k_scs_sum<<<kCols, 32, 0, st>>>(d_part.as<double>(), nblk, 1, d_sums.as<double>());
        k_scs_alpha<<<1, kCols, 0, st>>>(d_sums.as<double>(), st_d, d_flag.as<int>());
        k_scs_update<<<nblk, kWarps * 32, 0, st>>>(N, 0, st_d, d_p.as<double>(), d_q.as<double>(),
                                                   d_aiu_c.as<double>(), d_x.as<double>(), d_r.as<double>(),
                                                   d_part.as<double>(), nblk);
        k_scs_sum<<<2 * kCols, 32, 0, st>>>(d_part.as<double>(), nblk, 2, d_sums.as<double>());
        k_scs_beta<<<1, kCols, 0, st>>>(d_sums.as<double>(), st_d, 0);
        k_scs_direction<T><<<vgrid, 256, 0, st>>>(N, 1, st_d, d_r.as<double>(), d_aiu_c.as<double>(),
                                                  d_p.as<double>(), d_pT.as<T>());
        MBD_LAUNCH_CHECK();
        ++iters;
        MBD_TRY(residual(done));
    }
    int flag = 0;
    MBD_CUDA_TRY(cudaMemcpyAsync(&flag, d_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
    k_scs_finish<<<(N + 127) / 128, 128, 0, st>>>(N, ncol, d_x.as<double>(), d_al.as<double>(), a.rvdw,
                                                  d_wq.as<double>(), d_out.as<double>(), d_aiu.as<double>());
    MBD_LAUNCH_CHECK();
    std::vector<double> out(4 * (size_t)N), aiu(aiu_out ? (size_t)ncol * N : 0);
    MBD_CUDA_TRY(cudaMemcpyAsync(out.data(), d_out.ptr, out.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (aiu_out)
        MBD_CUDA_TRY(cudaMemcpyAsync(aiu.data(), d_aiu.ptr, aiu.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    MBD_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag) return MBD_ERR_NOT_POSITIVE_DEFINITE;
    for (double v : out)
        if (!std::isfinite(v)) return MBD_ERR_NONFINITE;
    for (double v : aiu)
        if (!std::isfinite(v)) return MBD_ERR_NONFINITE;
    std::copy(out.begin(), out.begin() + N, alpha_out);
    std::copy(out.begin() + N, out.begin() + 2 * N, omega_out);
    std::copy(out.begin() + 2 * N, out.begin() + 3 * N, rvdw_out);
    if (c6_out) std::copy(out.begin() + 3 * N, out.end(), c6_out);
    if (aiu_out) std::copy(aiu.begin(), aiu.end(), aiu_out);
    if (iters_out) *iters_out = iters;
    if (res_out) *res_out = worst;
    return MBD_OK;
}

}  // namespace
}  // namespace mbd

extern "C" mbd_status mbd_scs_screen(mbd_system *s, int32_t n_freq, double tol, int32_t max_iter, double *alpha_out,
                                     double *omega_out, double *r_vdw_out, double *c6_out, double *alpha_iu_out,
                                     int32_t *iterations, double *residual) {
    if (!s || !alpha_out || !omega_out || !r_vdw_out) return MBD_ERR_INVALID_ARG;
    if (n_freq < 1 || n_freq > 31 || !(tol > 0.0) || !std::isfinite(tol) || max_iter < 0 || max_iter > 100000)
        return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64)
        return mbd::screen<double>(s, n_freq, tol, max_iter, alpha_out, omega_out, r_vdw_out, c6_out, alpha_iu_out,
                                   iterations, residual);
    return mbd::screen<float>(s, n_freq, tol, max_iter, alpha_out, omega_out, r_vdw_out, c6_out, alpha_iu_out,
                              iterations, residual);
}
