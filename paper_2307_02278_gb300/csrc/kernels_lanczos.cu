// Lanczos-layer kernels (FP64): probe generation (Eq. dds), the recurrence
// prologue y*_k = l_{k-1} - a_{k-1} y_{k-1} - b_{k-1} y_{k-2}, b_k = ||y*_k||
// (Eq. recurs2, Algorithm 2), the tridiagonal Gauss quadrature (Eqs. tridiag2,
// sl3, sl4) and the trace/energy reduction (Eq. plasmonic2, Algorithm 1).
#include "mbd_internal.cuh"
#include "ql.cuh"

namespace mbd {

namespace {

// SplitMix64 (Steele, Lea & Flood 2014): first output for initial state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// u_{l,i} = +1 if the top bit of SplitMix64(seed + (l << 32) + i) is 0, else -1.
__device__ __forceinline__ double rademacher(uint64_t seed, uint64_t l, uint64_t i) {
    return (splitmix64(seed + (l << 32) + i) >> 63) ? -1.0 : 1.0;
}

template <class D>
__global__ void __launch_bounds__(256) k_prologue(LanczosView lz, int k, int m, uint64_t seed,
                                                  const uint64_t *__restrict__ seed_dev, int R, int ld, int rows,
                                                  const double *__restrict__ g, D *__restrict__ dout) {
    pdl_launch_dependents();
    pdl_wait();
    if (k == 0 && seed_dev != nullptr) seed = *seed_dev;   // replayed graphs read the seed from device memory
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < R;
    const size_t stride = (size_t)rows * ld;
    double *Yk = lz.Y + lz_slot(lz, k) * stride;
    double acc = 0.0;
    if (valid) {
        const double ak1 = k >= 1 ? lz.a[(size_t)(k - 1) * ld + r] : 0.0;
        const double bk2 = k >= 2 ? lz.b[(size_t)(k - 2) * ld + r] : 0.0;
        const double *Yk1 = k >= 1 ? lz.Y + lz_slot(lz, k - 1) * stride : nullptr;
        const double *Yk2 = k >= 2 ? lz.Y + lz_slot(lz, k - 2) * stride : nullptr;
        const double nrm0 = sqrt((double)rows);
        // four rows per iteration, all their loads issued before any use, so
        // that enough bytes are in flight to stream the FP64 vectors from HBM
        constexpr int UR = 4;
        const int rstep = gridDim.x * 8;
        for (int row0 = blockIdx.x * 8 + ty; row0 < rows; row0 += UR * rstep) {
            double lv[UR], y1[UR], y2[UR], gv[UR];
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                const int row = row0 + u * rstep;
                lv[u] = y1[u] = y2[u] = gv[u] = 0.0;
                if (row < rows) {
                    const size_t o = (size_t)row * ld + r;
                    gv[u] = g[row / 3];
                    if (k >= 1) {
                        lv[u] = lz.L[o];
                        y1[u] = Yk1[o];
                    }
                    if (k >= 2) y2[u] = Yk2[o];
                }
            }
#pragma unroll
            for (int u = 0; u < UR; ++u) {
                const int row = row0 + u * rstep;
                if (row < rows) {
                    const size_t o = (size_t)row * ld + r;
                    double ys;
                    if (k == 0) {
                        ys = rademacher(seed, (uint64_t)r, (uint64_t)row) / nrm0;
                    } else {
                        ys = lv[u] - ak1 * y1[u];
                        if (k >= 2) ys -= bk2 * y2[u];
                    }
                    Yk[o] = ys;
                    dout[o] = D(gv[u] * ys);
                    acc += ys * ys;
                }
            }
        }
    }
    __shared__ double red[8][32];
    __shared__ double bval[32], tot[32];
    red[ty][lane] = acc;
    __syncthreads();
    if (ty == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][lane];
        bval[lane] = s;
    }
    __syncthreads();
    if (grid_reduce(bval, 32, blockIdx.y * 32, R, ld, lz, tot) && ty == 0 && valid) {
        if (k == 0) {
            lz.invb[r] = 1.0;
            lz.length[r] = m;
        } else {
            double nrm = sqrt(tot[lane]);
            bool active = lz.length[r] == m;
            if (active && !(nrm > kBreakdown * fabs(lz.a[r]))) {
                lz.length[r] = k;
                active = false;
            }
            if (!active) nrm = 0.0;
            lz.b[(size_t)(k - 1) * ld + r] = nrm;
            lz.invb[r] = active ? 1.0 / nrm : 0.0;
        }
    }
}

// ---------------------------------------------------------------- Chebyshev quadrature
// The Gauss quadrature of probe l (Eqs. tridiag2, sl3) is
//   q_l = sum_k U_1k^2 sqrt(theta_k) = e_1^T Delta^{1/2} e_1,
// and the force estimator's coefficients are c = U diag(theta^{-1/2}) U^T e_1 =
// Delta^{-1/2} e_1.  Both are functions of Delta applied to e_1, so they need
// no eigendecomposition: with [L, U] containing the spectrum of Delta,
//   f(Delta) e_1 = sum_{j<N} c_j(f) T_j(X) e_1,  X = (Delta - mid I) / half,
// with Chebyshev coefficients c_j(f) of f(mid + half xi) on [-1, 1] (error
// decaying like rho^-N, rho = (sqrt(kappa) + 1) / (sqrt(kappa) - 1), kappa =
// U / L).  One warp per probe; rows are spread over the lanes (row k in lane
// k mod 32, register slot k / 32), so every step of the three-term recurrence
// is one tridiagonal product with two shuffles.
//   U: Gershgorin's upper bound.  L: two rounds of 32-way multisection with
//   Sturm counts (the number of eigenvalues below x, from the signs of the
//   characteristic polynomials of the leading blocks, rescaled to stay in
//   range); L has count 0, so L <= theta_min.  A count > 0 at x = 0 means a
//   non-positive Ritz value (status bit 1).
// Probes with L <= 0 or kappa too large for kChebMax terms are flagged in
// fallback[] for the QL kernel.  status bit 4: NaN/Inf in Delta.
constexpr int kChebMax = 256;
constexpr int kRowSlots = (kMaxSteps + 31) / 32;

__device__ int sturm_count(const double *a, const double *b2, int n, double x) {
    double pm = 1.0, p = a[0] - x;
    int cnt = p < 0.0 ? 1 : 0;
    for (int k = 1; k < n; ++k) {
        double pn = (a[k] - x) * p - b2[k - 1] * pm;
        if (pn == 0.0) pn = p < 0.0 ? 1e-300 : -1e-300;   // a zero is taken as a sign change
        cnt += ((pn < 0.0) != (p < 0.0)) ? 1 : 0;
        pm = p;
        p = pn;
        const double ap = fabs(p);
        if (ap > 1e150) {
            p *= 1e-150;
            pm *= 1e-150;
        } else if (ap < 1e-150 && fabs(pm) < 1e-150) {
            p *= 1e150;
            pm *= 1e150;
        }
    }
    return cnt;
}

template <bool FULL>
__global__ void __launch_bounds__(32) k_quad_cheb(const double *__restrict__ a, const double *__restrict__ b,
                                                  const int *__restrict__ length, int R, int ld, int m,
                                                  double *__restrict__ q, double *__restrict__ coef,
                                                  int *__restrict__ status, int *__restrict__ fallback) {
    __shared__ double sa[kMaxSteps], sb2[kMaxSteps], tab[4 * kChebMax], f1[kChebMax], f2[kChebMax];
    __shared__ double c1[kChebMax], c2[kChebMax];
    const int r = blockIdx.x, lane = threadIdx.x;
    const int n = length ? length[r] : m;
    // rows in registers: row k = lane + 32 t
    double ar[kRowSlots], br[kRowSlots], bl[kRowSlots];
    int finite = 1;
    double glo = 1e300, ghi = -1e300;
#pragma unroll
    for (int t = 0; t < kRowSlots; ++t) {
        const int k = lane + 32 * t;
        ar[t] = br[t] = 0.0;
        if (k < n) {
            ar[t] = a[(size_t)k * ld + r];
            br[t] = k < n - 1 ? b[(size_t)k * ld + r] : 0.0;
            finite &= (isfinite(ar[t]) && isfinite(br[t])) ? 1 : 0;
            sa[k] = ar[t];
            sb2[k] = br[t] * br[t];
        }
    }
#pragma unroll
    for (int t = 0; t < kRowSlots; ++t) {
        // b_{k-1}: lane - 1 of the same slot, or lane 31 of the previous one
        const double up = __shfl_up_sync(0xffffffffu, br[t], 1);
        const double prev31 = __shfl_sync(0xffffffffu, t > 0 ? br[t > 0 ? t - 1 : 0] : 0.0, 31);
        bl[t] = lane > 0 ? up : (t > 0 ? prev31 : 0.0);
        const int k = lane + 32 * t;
        if (k < n) {
            const double rad = fabs(bl[t]) + fabs(br[t]);
            glo = fmin(glo, ar[t] - rad);
            ghi = fmax(ghi, ar[t] + rad);
        }
    }
    finite = __all_sync(0xffffffffu, finite);
    for (int off = 16; off > 0; off >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, off));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
    }
    __syncwarp();
    if (!finite) {
        if (lane == 0) {
            atomicOr(status, 4);
            q[r] = 0.0;
            fallback[r] = 0;
        }
        if (FULL)
            for (int k = lane; k < m; k += 32) coef[(size_t)k * ld + r] = 0.0;
        return;
    }
    // ---- spectrum bracket [L, U]
    double lo = fmax(glo, 0.0), hi = ghi;
    bool pd = true;
    if (glo <= 0.0) {
        int c0 = lane == 0 ? sturm_count(sa, sb2, n, 0.0) : 0;
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        pd = c0 == 0;
    }
    if (pd) {
        for (int round = 0; round < 2; ++round) {
            const double x = lo + (hi - lo) * (double)(lane + 1) / 32.0;
            const int c = lane == 31 ? n : sturm_count(sa, sb2, n, x);   // hi: every eigenvalue below
            const unsigned bal = __ballot_sync(0xffffffffu, c >= 1);
            const int j = __ffs(bal) - 1;
            const double nlo = j == 0 ? lo : lo + (hi - lo) * (double)j / 32.0;
            const double nhi = lo + (hi - lo) * (double)(j + 1) / 32.0;
            lo = nlo;
            hi = nhi;
        }
    }
    // widened by a relative 1e-13 so that the interval has a width even when a
    // bound is an eigenvalue (a 1 x 1 Delta, a decoupled diagonal)
    const double L = lo * (1.0 - 1e-13), U = ghi * (1.0 + 1e-13) + 1e-300;
    int N = 0;
    if (pd && L > 0.0) {
        const double kap = U / L, sk = sqrt(kap);
        const double lrho = log((sk + 1.0) / (sk - 1.0));
        const double need = (log(1e17) + log(kap)) / lrho + 8.0;
        N = 32;
        while (N < need && N <= kChebMax) N *= 2;
    }
    if (!pd || N == 0 || N > kChebMax) {
        // non-positive definite (bit 1, as the QL kernel), or the expansion cannot
        // reach FP64 accuracy: QL takes the probe
        if (lane == 0) {
            if (!pd) atomicOr(status, 1);
            q[r] = 0.0;
            fallback[r] = pd ? 1 : 0;
        }
        if (FULL)
            for (int k = lane; k < m; k += 32) coef[(size_t)k * ld + r] = 0.0;
        return;
    }
    // ---- coefficients: c_j = (2/N) sum_i f(x_i) cos(pi j (i + 1/2) / N), x_i = mid + half cos(pi (i + 1/2) / N)
    const double mid = 0.5 * (U + L), half = 0.5 * (U - L);
    const int N4 = 4 * N;
    for (int k = lane; k < N4; k += 32) tab[k] = cospi((double)k / (2.0 * N));
    __syncwarp();
    for (int i = lane; i < N; i += 32) {
        const double x = mid + half * tab[2 * i + 1];
        const double sx = sqrt(x);
        f1[i] = sx;
        f2[i] = 1.0 / sx;
    }
    __syncwarp();
    for (int j = lane; j < N; j += 32) {
        double s1[4] = {0.0, 0.0, 0.0, 0.0}, s2[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < N; i += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double cv = tab[(j * (2 * (i + u) + 1)) & (N4 - 1)];
                s1[u] += f1[i + u] * cv;
                s2[u] += f2[i + u] * cv;
            }
        }
        const double sc = (j == 0 ? 1.0 : 2.0) / N;     // c_0 / 2 for the j = 0 term
        c1[j] = sc * ((s1[0] + s1[1]) + (s1[2] + s1[3]));
        c2[j] = sc * ((s2[0] + s2[1]) + (s2[2] + s2[3]));
    }
    __syncwarp();
    // ---- recurrence v_{j+1} = 2 X v_j - v_{j-1}, v_0 = e_1, accumulating sum c_j v_j
    const double ih = 1.0 / half;
    double am[kRowSlots], v0[kRowSlots], v1[kRowSlots], w[kRowSlots];
#pragma unroll
    for (int t = 0; t < kRowSlots; ++t) {
        const int k = lane + 32 * t;
        am[t] = k < n ? ar[t] - mid : 0.0;
        v0[t] = k == 0 ? 1.0 : 0.0;
        w[t] = c2[0] * v0[t];
    }
    double qa = c1[0];
    // v1 = X e_1
    auto matvec = [&](const double *v, double *y) {
#pragma unroll
        for (int t = 0; t < kRowSlots; ++t) {
            const double left0 = __shfl_up_sync(0xffffffffu, v[t], 1);
            const double l31 = __shfl_sync(0xffffffffu, v[t > 0 ? t - 1 : 0], 31);
            const double right0 = __shfl_down_sync(0xffffffffu, v[t], 1);
            const double r0 = __shfl_sync(0xffffffffu, v[t + 1 < kRowSlots ? t + 1 : t], 0);
            const double left = lane > 0 ? left0 : (t > 0 ? l31 : 0.0);
            const double right = lane < 31 ? right0 : (t + 1 < kRowSlots ? r0 : 0.0);
            y[t] = (am[t] * v[t] + bl[t] * left + br[t] * right) * ih;
        }
    };
    matvec(v0, v1);
#pragma unroll
    for (int t = 0; t < kRowSlots; ++t) w[t] += c2[1] * v1[t];
    qa += c1[1] * __shfl_sync(0xffffffffu, v1[0], 0);
    for (int j = 2; j < N; ++j) {
        double y[kRowSlots];
        matvec(v1, y);
#pragma unroll
        for (int t = 0; t < kRowSlots; ++t) {
            const double vn = 2.0 * y[t] - v0[t];
            v0[t] = v1[t];
            v1[t] = vn;
            w[t] += c2[j] * vn;
        }
        qa += c1[j] * __shfl_sync(0xffffffffu, v1[0], 0);
    }
    if (lane == 0) {
        q[r] = qa;
        fallback[r] = 0;
    }
    if (FULL) {
#pragma unroll
        for (int t = 0; t < kRowSlots; ++t) {
            const int k = lane + 32 * t;
            if (k < m) coef[(size_t)k * ld + r] = k < n ? w[t] : 0.0;
        }
    }
}

// Gauss quadrature of one probe's tridiagonal Delta (Eqs. tridiag2, sl3) by
// implicit QL (ql.cuh), one block of two warps per probe.  Warp 0 runs the
// sweeps (their scalar chain on lane 0) and records each sweep's rotations;
// warp 1 applies the previous sweep's rotations to the rows of U (I at the
// start) at the same time: rotations are double-buffered, one barrier per
// sweep.  The Gauss weights are U_1k^2, so without FULL only row 1 of U is
// kept; with FULL the whole U is kept and c = Delta^{-1/2} e_1 =
// U diag(theta^{-1/2}) U^T e_1 is returned as well (w = C^{-1/2} v =
// sum_k c_k y_k for the force estimator).  S = double (FP64) or df.
// status bit 1: a Ritz value <= 0; bit 2: a sweep limit hit; bit 4: NaN/Inf.
template <class S, bool FULL>
__global__ void __launch_bounds__(64) k_tridiag(const double *__restrict__ a, const double *__restrict__ b,
                                                const int *__restrict__ length, int R, int ld, int m,
                                                double *__restrict__ q, double *__restrict__ coef,
                                                int *__restrict__ status, const int *__restrict__ only) {
    if (only != nullptr && only[blockIdx.x] == 0) return;   // this probe was done by the Chebyshev kernel
    extern __shared__ __align__(16) unsigned char sm_raw[];
    S *d = reinterpret_cast<S *>(sm_raw);
    S *e = d + m;
    S *cs = e + m;          // [2][m]
    S *sn = cs + 2 * m;     // [2][m]
    S *Z = sn + 2 * m;      // [nz][n + 1]
    __shared__ int s_mm[2], s_nrot[2], s_done, s_bad;
    __shared__ double s_part[2];
    __shared__ int s_neg[2];
    const int r = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = length ? length[r] : m;
    const int zs = n + 1;
    const int nz = FULL ? n : 1;
    int finite = 1;
    for (int k2 = tid; k2 < n; k2 += 64) {
        const double dv = a[(size_t)k2 * ld + r];
        const double ev = (k2 < n - 1) ? b[(size_t)k2 * ld + r] : 0.0;
        finite &= (isfinite(dv) && isfinite(ev)) ? 1 : 0;
        to_scalar(dv, d[k2]);
        to_scalar(ev, e[k2]);
    }
    for (int row = tid; row < nz; row += 64)
        for (int col = 0; col < n; ++col) to_scalar(row == col ? 1.0 : 0.0, Z[row * zs + col]);
    if (tid == 0) {
        s_done = 0;
        s_bad = 0;
        s_nrot[0] = s_nrot[1] = 0;
    }
    finite = __syncthreads_and(finite);
    if (!finite) {
        if (tid == 0) {
            atomicOr(status, 4);
            q[r] = 0.0;
        }
        if (FULL)
            for (int k2 = tid; k2 < m; k2 += 64) coef[(size_t)k2 * ld + r] = 0.0;
        return;
    }
    int l = 0, iter = 0;        // warp-0 state (identical in its lanes)
    for (int t = 0;; ++t) {
        const int buf = t & 1;
        if (warp == 0) {
            bool produced = false;
            while (l < n && !produced) {
                const int mm = find_split(d, e, l, n);
                if (mm == l) {
                    ++l;
                    iter = 0;
                    continue;
                }
                if (++iter > 60) {
                    if (lane == 0) s_bad = 1;
                    l = n;
                    break;
                }
                __syncwarp();   // every lane has read d, e before lane 0 rewrites them
                if (lane == 0) {
                    int nrot = ql_sweep(d, e, cs + buf * m, sn + buf * m, l, mm);
                    if (nrot < 0) nrot = -nrot - 1;
                    s_nrot[buf] = nrot;
                    s_mm[buf] = mm;
                }
                __syncwarp();
                produced = true;
            }
            if (!produced && lane == 0) {
                s_nrot[buf] = 0;
                s_done = 1;
            }
        } else if (t > 0) {
            const int pb = buf ^ 1;
            const int nrot = s_nrot[pb], mm = s_mm[pb];
            if (nrot > 0)
                for (int row = lane; row < nz; row += 32)
                    apply_rotations(Z + row * zs, cs + pb * m, sn + pb * m, mm, nrot);
        }
        __syncthreads();
        if (s_done) break;      // the last sweep was applied in this pass
    }
    // q = sum_k U_1k^2 sqrt(theta_k)
    double part = 0.0;
    int neg = 0;
    for (int k2 = tid; k2 < n; k2 += 64) {
        const double th = from_scalar(d[k2]);
        const double z0 = from_scalar(Z[k2]);
        if (th > 0.0)
            part += z0 * z0 * sqrt(th);
        else
            neg = 1;
    }
    for (int off = 16; off > 0; off >>= 1) {
        part += __shfl_down_sync(0xffffffffu, part, off);
        neg |= __shfl_down_sync(0xffffffffu, neg, off);
    }
    if (lane == 0) {
        s_part[warp] = part;
        s_neg[warp] = neg;
    }
    __syncthreads();
    if (tid == 0) {
        q[r] = s_part[0] + s_part[1];
        if (s_neg[0] | s_neg[1]) atomicOr(status, 1);
        if (s_bad) atomicOr(status, 2);
    }
    if (FULL) {
        // c_k = sum_j U_kj theta_j^{-1/2} U_1j
        for (int k2 = tid; k2 < m; k2 += 64) {
            double c = 0.0;
            if (k2 < n)
                for (int j = 0; j < n; ++j) {
                    const double th = from_scalar(d[j]);
                    if (th > 0.0) c += from_scalar(Z[k2 * zs + j]) * from_scalar(Z[j]) * rsqrt(th);
                }
            coef[(size_t)k2 * ld + r] = c;
        }
    }
}

// Tr sqrt(C) ~ (D/R) sum_l q_l; E = 0.5 Tr - 1.5 sum w.  One block, fixed order.
__global__ void k_energy_reduce(const double *__restrict__ q, int R, int dim, double omega_sum,
                                double *__restrict__ scal) {
    __shared__ double red[256];
    double s = 0.0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) s += q[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double tr = (double)dim / (double)R * red[0];
        scal[0] = 0.5 * tr - 1.5 * omega_sum;
        scal[1] = tr;
    }
}

__global__ void k_probes(uint64_t seed, int first, int R, int dim, double *__restrict__ v) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)R * dim) return;
    const int l = (int)(idx / dim), i = (int)(idx % dim);
    v[idx] = rademacher(seed, (uint64_t)(first + l), (uint64_t)i) / sqrt((double)dim);
}

// Dense-operator Lanczos step (for checking the Lanczos layer alone):
// L = (C y*) / b, one warp per row, lane = probe.
__global__ void __launch_bounds__(256) k_dense_matvec(const double *__restrict__ c, int dim, LanczosView lz, int k,
                                                      int R, int ld) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y * 32 + lane;
    const int row = blockIdx.x * 8 + warp;
    if (row >= dim || r >= R) return;
    const double *Yk = lz.Y + lz_slot(lz, k) * dim * ld;
    double s = 0.0;
    for (int col = 0; col < dim; ++col) s += c[(size_t)row * dim + col] * Yk[(size_t)col * ld + r];
    lz.L[(size_t)row * ld + r] = s * lz.invb[r];
}

__global__ void __launch_bounds__(256) k_dense_epilogue(int dim, LanczosView lz, int k, int R, int ld) {
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < R;
    double *Yk = lz.Y + lz_slot(lz, k) * dim * ld;
    double acc = 0.0;
    if (valid) {
        const double ib = lz.invb[r];
        for (int row = blockIdx.x * 8 + ty; row < dim; row += gridDim.x * 8) {
            const size_t o = (size_t)row * ld + r;
            const double y = Yk[o] * ib;
            Yk[o] = y;
            acc += y * lz.L[o];
        }
    }
    __shared__ double red[8][32];
    __shared__ double bval[32], tot[32];
    red[ty][lane] = acc;
    __syncthreads();
    if (ty == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][lane];
        bval[lane] = s;
    }
    __syncthreads();
    if (grid_reduce(bval, 32, blockIdx.y * 32, R, ld, lz, tot) && ty == 0 && valid)
        lz.a[(size_t)k * ld + r] = tot[lane];
}

// [nvec][rows] <-> [rows][ld] transposes through a 32x33 shared tile.
__global__ void k_transpose_in(const double *__restrict__ x, int nvec, int rows, double *__restrict__ xt, int ld) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, v0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int v = v0 + j, row = r0 + threadIdx.x;
        tile[j][threadIdx.x] = (v < nvec && row < rows) ? x[(size_t)v * rows + row] : 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int row = r0 + j, v = v0 + threadIdx.x;
        if (row < rows && v < ld) xt[(size_t)row * ld + v] = tile[threadIdx.x][j];
    }
}
__global__ void k_transpose_out(const double *__restrict__ xt, int nvec, int rows, int ld, double *__restrict__ x) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, v0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int row = r0 + j, v = v0 + threadIdx.x;
        tile[j][threadIdx.x] = (row < rows && v < nvec) ? xt[(size_t)row * ld + v] : 0.0;
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int v = v0 + j, row = r0 + threadIdx.x;
        if (v < nvec && row < rows) x[(size_t)v * rows + row] = tile[threadIdx.x][j];
    }
}
template <class T> __global__ void k_cast(const double *__restrict__ x, T *__restrict__ y, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = T(x[i]);
}
// d = g . x (per row, g indexed by atom = row / 3), cast to T
template <class T>
__global__ void k_gscale(const double *__restrict__ x, const double *__restrict__ g, T *__restrict__ d, int rows,
                         int ld) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)rows * ld) return;
    d[i] = T(g[(i / ld) / 3] * x[i]);
}
template <class T>
__global__ void k_mesh_out(const T *__restrict__ mesh, int nvec, size_t npts, int ld, double *__restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts * nvec) return;
    const size_t v = i / npts, pt = i % npts;
    out[i] = double(mesh[pt * ld + v]);
}
template <class T>
__global__ void k_mesh_in(const double *__restrict__ in, int nvec, size_t npts, int ld, T *__restrict__ mesh) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts * ld) return;
    const size_t pt = i / ld, v = i % ld;
    mesh[i] = v < (size_t)nvec ? T(in[v * npts + pt]) : T(0);
}

}  // namespace

int probe_ld(int R) { return R + (R & 1); }

mbd_status launch_prologue_t(cudaStream_t st, const LanczosView &lz, int k, int m, uint64_t seed, int R, int ld,
                             int rows, const double *g, void *dout, int dtype_bytes, int nblk,
                             const uint64_t *seed_dev) {
    dim3 block(32, 8), grid(nblk, (R + 31) / 32);
    if (dtype_bytes == 8)
        k_prologue<double><<<grid, block, 0, st>>>(lz, k, m, seed, seed_dev, R, ld, rows, g,
                                                   static_cast<double *>(dout));
    else
        k_prologue<float><<<grid, block, 0, st>>>(lz, k, m, seed, seed_dev, R, ld, rows, g,
                                                  static_cast<float *>(dout));
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class S>
mbd_status launch_tridiag_s(const double *a, const double *b, const int *length, int R, int ld, int m, double *q,
                            double *coef, int *status, cudaStream_t st, const int *only) {
    const bool full = coef != nullptr;
    const size_t smem = sizeof(S) * (size_t)(6 * m + (full ? m * (m + 1) : m + 1));
    if (full) {
        if (smem > 48 * 1024)
            MBD_CUDA_TRY(cudaFuncSetAttribute(k_tridiag<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_tridiag<S, true><<<R, 64, smem, st>>>(a, b, length, R, ld, m, q, coef, status, only);
    } else {
        k_tridiag<S, false><<<R, 64, smem, st>>>(a, b, length, R, ld, m, q, nullptr, status, only);
    }
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_quadrature(const double *a, const double *b, const int *length, int R, int ld, int m, double *q,
                             double *coef, int *status, int *fallback, cudaStream_t st, int method) {
    if (method == MBD_QUAD_QL_DF64) return launch_tridiag_s<df>(a, b, length, R, ld, m, q, coef, status, st, nullptr);
    if (method == MBD_QUAD_QL) return launch_tridiag_s<double>(a, b, length, R, ld, m, q, coef, status, st, nullptr);
    if (coef)
        k_quad_cheb<true><<<R, 32, 0, st>>>(a, b, length, R, ld, m, q, coef, status, fallback);
    else
        k_quad_cheb<false><<<R, 32, 0, st>>>(a, b, length, R, ld, m, q, coef, status, fallback);
    MBD_LAUNCH_CHECK();
    // probes whose spectrum the expansion cannot cover go through QL
    return launch_tridiag_s<double>(a, b, length, R, ld, m, q, coef, status, st, fallback);
}

mbd_status launch_energy_reduce(const double *q, int R, int dim, double omega_sum, double *scal, cudaStream_t st) {
    k_energy_reduce<<<1, 256, 0, st>>>(q, R, dim, omega_sum, scal);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_probes(uint64_t seed, int first, int R, int dim, double *v, cudaStream_t st) {
    const size_t n = (size_t)R * dim;
    k_probes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, first, R, dim, v);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_dense_step(const double *c, int dim, const LanczosView &lz, int k, int R, int ld, int nblk,
                             cudaStream_t st) {
    dim3 g1((dim + 7) / 8, (R + 31) / 32);
    k_dense_matvec<<<g1, 256, 0, st>>>(c, dim, lz, k, R, ld);
    MBD_LAUNCH_CHECK();
    dim3 g2(nblk, (R + 31) / 32), b2(32, 8);
    k_dense_epilogue<<<g2, b2, 0, st>>>(dim, lz, k, R, ld);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_to_probe_major(const double *x, int nvec, int rows, double *xt, int ld, cudaStream_t st) {
    dim3 grid((rows + 31) / 32, (ld + 31) / 32), block(32, 8);
    k_transpose_in<<<grid, block, 0, st>>>(x, nvec, rows, xt, ld);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
mbd_status launch_from_probe_major(const double *xt, int nvec, int rows, int ld, double *x, cudaStream_t st) {
    dim3 grid((rows + 31) / 32, (nvec + 31) / 32), block(32, 8);
    k_transpose_out<<<grid, block, 0, st>>>(xt, nvec, rows, ld, x);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
template <class T> mbd_status launch_cast_rows(const double *x, T *y, size_t n, cudaStream_t st) {
    k_cast<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, n);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
template <class T>
mbd_status launch_mesh_out(const T *mesh, int nvec, size_t npts, int ld, double *out, cudaStream_t st) {
    const size_t n = npts * nvec;
    k_mesh_out<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mesh, nvec, npts, ld, out);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
template <class T>
mbd_status launch_mesh_in(const double *in, int nvec, size_t npts, int ld, T *mesh, cudaStream_t st) {
    const size_t n = npts * ld;
    k_mesh_in<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, nvec, npts, ld, mesh);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T> mbd_status launch_gscale(const double *x, const double *g, T *d, int rows, int ld, cudaStream_t st) {
    const size_t n = (size_t)rows * ld;
    k_gscale<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, g, d, rows, ld);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
template mbd_status launch_gscale<double>(const double *, const double *, double *, int, int, cudaStream_t);
template mbd_status launch_gscale<float>(const double *, const double *, float *, int, int, cudaStream_t);
template mbd_status launch_cast_rows<double>(const double *, double *, size_t, cudaStream_t);
template mbd_status launch_cast_rows<float>(const double *, float *, size_t, cudaStream_t);
template mbd_status launch_mesh_out<double>(const double *, int, size_t, int, double *, cudaStream_t);
template mbd_status launch_mesh_out<float>(const float *, int, size_t, int, double *, cudaStream_t);
template mbd_status launch_mesh_in<double>(const double *, int, size_t, int, double *, cudaStream_t);
template mbd_status launch_mesh_in<float>(const double *, int, size_t, int, float *, cudaStream_t);

}  // namespace mbd
