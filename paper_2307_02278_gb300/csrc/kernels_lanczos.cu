// Lanczos-layer kernels (FP64): probe generation (Eq. dds), the recurrence
// prologue y*_k = l_{k-1} - a_{k-1} y_{k-1} - b_{k-1} y_{k-2}, b_k = ||y*_k||
// (Eq. recurs2, Algorithm 2), the tridiagonal Gauss quadrature (Eqs. tridiag2,
// sl3, sl4) and the trace/energy reduction (Eq. plasmonic2, Algorithm 1).
#include "mbd_internal.cuh"

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
__global__ void __launch_bounds__(256) k_prologue(LanczosView lz, int k, int m, uint64_t seed, int R, int ld,
                                                  int rows, const double *__restrict__ g, D *__restrict__ dout) {
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < R;
    const size_t stride = (size_t)rows * ld;
    double *Yk = lz.Y + (size_t)k * stride;
    double acc = 0.0;
    if (valid) {
        const double ak1 = k >= 1 ? lz.a[(size_t)(k - 1) * ld + r] : 0.0;
        const double bk2 = k >= 2 ? lz.b[(size_t)(k - 2) * ld + r] : 0.0;
        const double *Yk1 = k >= 1 ? lz.Y + (size_t)(k - 1) * stride : nullptr;
        const double *Yk2 = k >= 2 ? lz.Y + (size_t)(k - 2) * stride : nullptr;
        const double nrm0 = sqrt((double)rows);
        for (int row = blockIdx.x * 8 + ty; row < rows; row += gridDim.x * 8) {
            const size_t o = (size_t)row * ld + r;
            double ys;
            if (k == 0) {
                ys = rademacher(seed, (uint64_t)r, (uint64_t)row) / nrm0;
            } else {
                ys = lz.L[o] - ak1 * Yk1[o];
                if (k >= 2) ys -= bk2 * Yk2[o];
            }
            Yk[o] = ys;
            dout[o] = D(g[row / 3] * ys);
            acc += ys * ys;
        }
    }
    __shared__ double red[8][32];
    __shared__ bool last;
    red[ty][lane] = acc;
    __syncthreads();
    if (ty == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][lane];
        if (valid) lz.partial[(size_t)blockIdx.x * ld + r] = s;
        __threadfence();
    }
    __syncthreads();
    if (lane == 0 && ty == 0) {
        const unsigned prev = atomicAdd(&lz.counter[blockIdx.y], 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && ty == 0) {
        __threadfence();
        if (valid) {
            if (k == 0) {
                lz.invb[r] = 1.0;
                lz.length[r] = m;
            } else {
                double s = 0.0;
                for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&lz.partial[(size_t)b * ld + r]);
                double nrm = sqrt(s);
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
        if (lane == 0) lz.counter[blockIdx.y] = 0u;
    }
}

// Implicit QL with Wilkinson shifts on a symmetric tridiagonal (diagonal d,
// sub-diagonal e; Bowdler, Martin, Reinsch & Wilkinson 1968).  Accumulates the
// plane rotations into the rows of Z selected by nz (nz = 1: the first row
// only, which is all the Gauss weights U_1k^2 need; Golub & Welsch 1969).
// Arrays are strided by `st` (probe-innermost scratch).  Returns false if an
// eigenvalue needs more than 60 sweeps.
__device__ bool ql_implicit(double *d, double *e, double *Z, int n, int nz, size_t st) {
    const double eps = 2.220446049250313e-16;
#define D_(i) d[(size_t)(i) * st]
#define E_(i) e[(size_t)(i) * st]
#define Z_(row, col) Z[((size_t)(row) * n + (col)) * st]
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        for (;;) {
            int mm = l;
            for (; mm < n - 1; ++mm) {
                const double dd = fabs(D_(mm)) + fabs(D_(mm + 1));
                if (fabs(E_(mm)) <= eps * dd) break;
            }
            if (mm == l) break;
            if (++iter > 60) return false;
            double g = (D_(l + 1) - D_(l)) / (2.0 * E_(l));
            double r = hypot(g, 1.0);
            g = D_(mm) - D_(l) + E_(l) / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            bool underflow = false;
            for (int i = mm - 1; i >= l; --i) {
                const double f = s * E_(i);
                const double b = c * E_(i);
                r = hypot(f, g);
                E_(i + 1) = r;
                if (r == 0.0) {
                    D_(i + 1) -= p;
                    E_(mm) = 0.0;
                    underflow = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = D_(i + 1) - p;
                r = (D_(i) - g) * s + 2.0 * c * b;
                p = s * r;
                D_(i + 1) = g + p;
                g = c * r - b;
                for (int row = 0; row < nz; ++row) {
                    const double zf = Z_(row, i + 1);
                    Z_(row, i + 1) = s * Z_(row, i) + c * zf;
                    Z_(row, i) = c * Z_(row, i) - s * zf;
                }
            }
            if (underflow) continue;
            D_(l) -= p;
            E_(l) = g;
            E_(mm) = 0.0;
        }
    }
#undef D_
#undef E_
#undef Z_
    return true;
}

// One thread per probe: q_l = sum_k U_1k^2 sqrt(theta_k).  status bit 1: a
// Ritz value <= 0; bit 2: no convergence; bit 4: non-finite input.
__global__ void k_quadrature(const double *__restrict__ a, const double *__restrict__ b,
                             const int *__restrict__ length, int R, int ld, int m, double *__restrict__ q,
                             int *__restrict__ status, double *__restrict__ work) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int n = length ? length[r] : m;
    const size_t st = (size_t)R;
    double *d = work + r, *e = work + (size_t)m * R + r, *z = work + (size_t)2 * m * R + r;
    bool finite = true;
    for (int k = 0; k < n; ++k) {
        d[k * st] = a[(size_t)k * ld + r];
        e[k * st] = (k < n - 1) ? b[(size_t)k * ld + r] : 0.0;
        z[k * st] = (k == 0) ? 1.0 : 0.0;
        finite = finite && isfinite(d[k * st]) && isfinite(e[k * st]);
    }
    if (!finite) {
        atomicOr(status, 4);
        q[r] = 0.0;
        return;
    }
    if (!ql_implicit(d, e, z, n, 1, st)) atomicOr(status, 2);
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        const double th = d[k * st];
        if (!(th > 0.0)) {
            atomicOr(status, 1);
            continue;
        }
        s += z[k * st] * z[k * st] * sqrt(th);
    }
    q[r] = s;
}

// Coefficients c = Delta^{-1/2} e_1 = U diag(theta^{-1/2}) U^T e_1 per probe
// (w = C^{-1/2} v ~ sum_k c_k y_k), full eigenvectors in scratch.
__global__ void k_inv_sqrt_coeffs(const double *__restrict__ a, const double *__restrict__ b,
                                  const int *__restrict__ length, int R, int ld, int m, double *__restrict__ coef,
                                  int *__restrict__ status, double *__restrict__ work) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const int n = length[r];
    const size_t st = (size_t)R;
    double *d = work + r, *e = work + (size_t)m * R + r, *Z = work + (size_t)2 * m * R + r;
    for (int k = 0; k < n; ++k) {
        d[k * st] = a[(size_t)k * ld + r];
        e[k * st] = (k < n - 1) ? b[(size_t)k * ld + r] : 0.0;
        for (int j = 0; j < n; ++j) Z[((size_t)k * n + j) * st] = (k == j) ? 1.0 : 0.0;
    }
    if (!ql_implicit(d, e, Z, n, n, st)) atomicOr(status, 2);
    for (int k = 0; k < m; ++k) {
        double s = 0.0;
        if (k < n) {
            for (int j = 0; j < n; ++j) {
                const double th = d[j * st];
                if (!(th > 0.0)) {
                    atomicOr(status, 1);
                    continue;
                }
                s += Z[((size_t)k * n + j) * st] * Z[(size_t)j * st] / sqrt(th);
            }
        }
        coef[(size_t)k * ld + r] = s;
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
    const double *Yk = lz.Y + (size_t)k * dim * ld;
    double s = 0.0;
    for (int col = 0; col < dim; ++col) s += c[(size_t)row * dim + col] * Yk[(size_t)col * ld + r];
    lz.L[(size_t)row * ld + r] = s * lz.invb[r];
}

__global__ void __launch_bounds__(256) k_dense_epilogue(int dim, LanczosView lz, int k, int R, int ld) {
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < R;
    double *Yk = lz.Y + (size_t)k * dim * ld;
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
    __shared__ bool last;
    red[ty][lane] = acc;
    __syncthreads();
    if (ty == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w][lane];
        if (valid) lz.partial[(size_t)blockIdx.x * ld + r] = s;
        __threadfence();
    }
    __syncthreads();
    if (lane == 0 && ty == 0) {
        const unsigned prev = atomicAdd(&lz.counter[blockIdx.y], 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && ty == 0) {
        __threadfence();
        double s = 0.0;
        if (valid)
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&lz.partial[(size_t)b * ld + r]);
        if (valid) lz.a[(size_t)k * ld + r] = s;
        if (lane == 0) lz.counter[blockIdx.y] = 0u;
    }
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
                             int rows, const double *g, void *dout, int dtype_bytes, int nblk) {
    dim3 block(32, 8), grid(nblk, (R + 31) / 32);
    if (dtype_bytes == 8)
        k_prologue<double><<<grid, block, 0, st>>>(lz, k, m, seed, R, ld, rows, g, static_cast<double *>(dout));
    else
        k_prologue<float><<<grid, block, 0, st>>>(lz, k, m, seed, R, ld, rows, g, static_cast<float *>(dout));
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_quadrature_t(const double *a, const double *b, const int *length, int R, int ld, int m, double *q,
                               int *status, double *work, cudaStream_t st) {
    k_quadrature<<<(R + 63) / 64, 64, 0, st>>>(a, b, length, R, ld, m, q, status, work);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

mbd_status launch_inv_sqrt_t(const double *a, const double *b, const int *length, int R, int ld, int m, double *coef,
                             int *status, double *work, cudaStream_t st) {
    k_inv_sqrt_coeffs<<<(R + 63) / 64, 64, 0, st>>>(a, b, length, R, ld, m, coef, status, work);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
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
