// Per-system setup kernels: real-space pair tensors, B-spline stencils and the
// SPME influence function.  These run once per geometry (mbd_create_system,
// mbd_update_positions), not per Lanczos step.
#include "mbd_internal.cuh"

#include <algorithm>
#include <cmath>

namespace mbd {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrtPi = 1.77245385090551602730;

// Radial coefficients of the real-space pair tensor A = c_id I - c_rr r r^T
// (Eq. fld_ewald with the damping correction) and of its derivative,
//   erfc part  c_id = B1, c_rr = B2 (Smith's B_n, (1/r) dB_n/dr = -B_{n+1})
//   damping    c_id -= (1 - s)/r^3, c_rr -= 3 (1 - s)/r^5,
// with cid_p = c_id'/r and crr_p = c_rr'/r.  FP64, with one reciprocal of r
// in place of the divisions by powers of r.
struct PairRadial {
    double cid, crr, cid_p, crr_p;
};
__device__ __forceinline__ PairRadial pair_radial(double r2, double rsum, double beta, double r_cut,
                                                  double damp_cut, double damp_beta, double damp_d) {
    PairRadial pr{0.0, 0.0, 0.0, 0.0};
    const double rho = sqrt(r2);
    const double inv_rho = 1.0 / rho, inv_r2 = inv_rho * inv_rho;
    if (rho < r_cut) {
        const double e = exp(-beta * beta * r2);
        const double b0 = erfc(beta * rho) * inv_rho;
        const double b1 = (b0 + 2.0 * beta / kSqrtPi * e) * inv_r2;
        const double b2 = (3.0 * b1 + 4.0 * beta * beta * beta / kSqrtPi * e) * inv_r2;
        const double b3 = (5.0 * b2 + 8.0 * beta * beta * beta * beta * beta / kSqrtPi * e) * inv_r2;
        pr.cid = b1;
        pr.crr = b2;
        pr.cid_p = -b2;
        pr.crr_p = -b3;
    }
    if (rho < damp_cut) {
        const double inv_R = 1.0 / (damp_beta * rsum);
        const double x = damp_d * (rho * inv_R - 1.0);
        const double oms = 1.0 / (1.0 + exp(x));          // 1 - s
        const double s = 1.0 - oms;
        const double dsdr = damp_d * inv_R * s * oms;
        const double inv_r3 = inv_r2 * inv_rho, inv_r5 = inv_r3 * inv_r2;
        // d/dr (oms / r^3) = -dsdr / r^3 - 3 oms / r^4 ;  d/dr (3 oms / r^5) = -3 dsdr / r^5 - 15 oms / r^6
        pr.cid -= oms * inv_r3;
        pr.crr -= 3.0 * oms * inv_r5;
        pr.cid_p -= (-dsdr * inv_r3 - 3.0 * oms * inv_r3 * inv_rho) * inv_rho;
        pr.crr_p -= (-3.0 * dsdr * inv_r5 - 15.0 * oms * inv_r5 * inv_rho) * inv_rho;
    }
    return pr;
}

// dA_ab / dr_c = cid_p r_c delta_ab - crr_p r_c r_a r_b - c_rr (delta_ac r_b + delta_bc r_a),
// (ab) over the 6 upper-triangle entries, c = x, y, z.
__device__ __forceinline__ void pair_tensor_grad(double rx, double ry, double rz, const PairRadial &pr,
                                                 double out[18]) {
    const double rv[3] = {rx, ry, rz};
    int o = 0;
    for (int ab = 0; ab < 6; ++ab) {
        const int ia = ab < 3 ? 0 : (ab < 5 ? 1 : 2);
        const int ib = ab < 3 ? ab : (ab < 5 ? ab - 2 : 2);
        for (int c = 0; c < 3; ++c) {
            double v = -pr.crr_p * rv[c] * rv[ia] * rv[ib];
            if (ia == ib) v += pr.cid_p * rv[c];
            if (ia == c) v -= pr.crr * rv[ib];
            if (ib == c) v -= pr.crr * rv[ia];
            out[o++] = v;
        }
    }
}

// Real-space pair tensor of E^dir with the damping correction (Eq. fld_ewald):
//   A(r) = [|r| < r_cut] (B1 I - B2 r r^T) - [|r| < damp_cut] (1 - s(|r|)) T(r)
// with Smith's erfc-screened B1, B2 and the bare T(r) = (r^2 I - 3 r r^T)/r^5,
// and its derivative dA/dr (forces).  FP64 from positions and the image shift,
// stored in T; a warp per atom, lanes over its neighbours.
template <class T>
__global__ void k_pair_tensors(int N, const double *__restrict__ pos, const double *__restrict__ rvdw,
                               const int *__restrict__ row, const int *__restrict__ col,
                               const int *__restrict__ shift, Geom g, double beta, double r_cut,
                               double damp_cut, double damp_beta, double damp_d, T *__restrict__ A,
                               T *__restrict__ dA, long long cap) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    const int nb1 = (int)min((long long)row[i + 1], cap);   // pairs beyond the buffers: rebuilt by the caller
    for (int nb = row[i] + lane; nb < nb1; nb += 32) {
        const int j = col[nb];
        const int sh = shift[nb];
        const double n1 = double((sh & 255) - 128), n2 = double(((sh >> 8) & 255) - 128),
                     n3 = double(((sh >> 16) & 255) - 128);
        const double rx = xi - pos[3 * j] - (n1 * g.cell[0] + n2 * g.cell[3] + n3 * g.cell[6]);
        const double ry = yi - pos[3 * j + 1] - (n1 * g.cell[1] + n2 * g.cell[4] + n3 * g.cell[7]);
        const double rz = zi - pos[3 * j + 2] - (n1 * g.cell[2] + n2 * g.cell[5] + n3 * g.cell[8]);
        const double r2 = rx * rx + ry * ry + rz * rz;
        const PairRadial pr = pair_radial(r2, rvdw[i] + rvdw[j], beta, r_cut, damp_cut, damp_beta, damp_d);
        T *a = A + 6 * (size_t)nb;
        a[0] = T(pr.cid - pr.crr * rx * rx);
        a[1] = T(-pr.crr * rx * ry);
        a[2] = T(-pr.crr * rx * rz);
        a[3] = T(pr.cid - pr.crr * ry * ry);
        a[4] = T(-pr.crr * ry * rz);
        a[5] = T(pr.cid - pr.crr * rz * rz);
        double gr[18];
        pair_tensor_grad(rx, ry, rz, pr, gr);
        T *ga = dA + 18 * (size_t)nb;
        for (int c = 0; c < 18; ++c) ga[c] = T(gr[c]);
    }
}

// Cardinal B-spline values on the stencil of one coordinate (Eq. scaledfractional):
// for x = frac(u) in [0,1), m[t] = M_p(x + t), dm[t] = M_p'(x + t), d2m[t] = M_p''(x + t),
// t = 0..p-1, from M_2 by the recursion M_n(y) = (y M_{n-1}(y) + (n - y) M_{n-1}(y - 1)) / (n - 1);
// M_n' = M_{n-1}(y) - M_{n-1}(y-1) and M_n'' = M_{n-2}(y) - 2 M_{n-2}(y-1) + M_{n-2}(y-2).
__device__ void bspline_stencil(double x, int p, double *m, double *dm, double *d2m) {
    double cur[kMaxOrder + 1], prev[kMaxOrder + 1], prev2[kMaxOrder + 1];
    for (int t = 0; t <= kMaxOrder; ++t) cur[t] = prev[t] = prev2[t] = 0.0;
    cur[0] = x;
    cur[1] = 1.0 - x;   // M_2(x), M_2(x+1)
    for (int n = 3; n <= p; ++n) {
        for (int t = 0; t <= kMaxOrder; ++t) {
            prev2[t] = prev[t];
            prev[t] = cur[t];
        }
        for (int t = 0; t < n; ++t) {
            const double y = x + t;
            const double hi = (t < n - 1) ? prev[t] : 0.0;
            const double lo = (t >= 1) ? prev[t - 1] : 0.0;
            cur[t] = (y * hi + (double(n) - y) * lo) / double(n - 1);
        }
    }
    // here cur = M_p, prev = M_{p-1}, prev2 = M_{p-2} (p >= 4)
    for (int t = 0; t < p; ++t) {
        m[t] = cur[t];
        dm[t] = prev[t] - (t >= 1 ? prev[t - 1] : 0.0);
        d2m[t] = prev2[t] - 2.0 * (t >= 1 ? prev2[t - 1] : 0.0) + (t >= 2 ? prev2[t - 2] : 0.0);
    }
}

// Per atom and dimension: u = K a*.R wrapped to [0, K), top = floor(u) and the
// stencil weights of mesh points top - t (mod K).
template <class T>
__global__ void k_splines(int N, const double *__restrict__ pos, Geom g, int *__restrict__ top,
                          T *__restrict__ w, T *__restrict__ dw, T *__restrict__ d2w, double *__restrict__ w64,
                          double *__restrict__ dw64) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * N) return;
    const int i = idx / 3, a = idx % 3;
    const int K = a == 0 ? g.K1 : (a == 1 ? g.K2 : g.K3);
    // recip row a = cmat row a / K
    const double u_raw = (g.cmat[3 * a] * pos[3 * i] + g.cmat[3 * a + 1] * pos[3 * i + 1] +
                          g.cmat[3 * a + 2] * pos[3 * i + 2]);
    double u = u_raw - floor(u_raw / K) * K;
    if (u >= K) u -= K;
    if (u < 0.0) u = 0.0;
    int t0 = (int)floor(u);
    if (t0 >= K) t0 = K - 1;
    const double x = u - t0;
    double m[kMaxOrder], dm[kMaxOrder], d2m[kMaxOrder];
    bspline_stencil(x, g.p, m, dm, d2m);
    top[idx] = t0;
    for (int t = 0; t < g.p; ++t) {
        w[(size_t)idx * g.p + t] = T(m[t]);
        dw[(size_t)idx * g.p + t] = T(dm[t]);
        d2w[(size_t)idx * g.p + t] = T(d2m[t]);
        w64[(size_t)idx * g.p + t] = m[t];
        dw64[(size_t)idx * g.p + t] = dm[t];
    }
}

// G(m) = B(m) exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), G(0) = 0 (tin-foil),
// m = sum_alpha m_alpha a*_alpha with the folded index (m = k for k <= K/2,
// else k - K), symmetrised with G(-m mod K).
__device__ double influence_at(int k1, int k2, int k3, Geom g, const double *bm1, const double *bm2,
                               const double *bm3, double beta, double vol) {
    if (k1 == 0 && k2 == 0 && k3 == 0) return 0.0;
    const int f1 = k1 <= g.K1 / 2 ? k1 : k1 - g.K1;
    const int f2 = k2 <= g.K2 / 2 ? k2 : k2 - g.K2;
    const int f3 = k3 <= g.K3 / 2 ? k3 : k3 - g.K3;
    // a*_alpha = cmat row alpha / K_alpha
    double mx = 0, my = 0, mz = 0;
    const double c1 = double(f1) / g.K1, c2 = double(f2) / g.K2, c3 = double(f3) / g.K3;
    mx = c1 * g.cmat[0] + c2 * g.cmat[3] + c3 * g.cmat[6];
    my = c1 * g.cmat[1] + c2 * g.cmat[4] + c3 * g.cmat[7];
    mz = c1 * g.cmat[2] + c2 * g.cmat[5] + c3 * g.cmat[8];
    const double m2 = mx * mx + my * my + mz * mz;
    return bm1[k1] * bm2[k2] * bm3[k3] * exp(-kPi * kPi * m2 / (beta * beta)) / (kPi * vol * m2);
}

template <class T>
__global__ void k_influence(Geom g, const double *__restrict__ bmod, double beta, double vol, T *__restrict__ G) {
    const size_t total = (size_t)g.K1 * g.K2 * g.K3;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int k3 = idx % g.K3;
    const int k2 = (idx / g.K3) % g.K2;
    const int k1 = idx / ((size_t)g.K2 * g.K3);
    const double *bm1 = bmod, *bm2 = bmod + g.K1, *bm3 = bmod + g.K1 + g.K2;
    const double gp = influence_at(k1, k2, k3, g, bm1, bm2, bm3, beta, vol);
    const double gn = influence_at((g.K1 - k1) % g.K1, (g.K2 - k2) % g.K2, (g.K3 - k3) % g.K3, g, bm1, bm2,
                                   bm3, beta, vol);
    G[idx] = T(0.5 * (gp + gn));
}

Geom make_geom(const mbd_system *s) {
    Geom g;
    g.N = s->N;
    g.K1 = s->K[0];
    g.K2 = s->K[1];
    g.K3 = s->K[2];
    g.p = s->p;
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) g.cmat[3 * b + a] = s->K[b] * s->recip[3 * b + a];
    for (int k = 0; k < 9; ++k) g.cell[k] = s->cell[k];
    return g;
}

// Real-space neighbour list over a cell grid (cells of width >= rmax along
// each reciprocal direction, kk cells searched each way).  A warp per atom i
// visits the cells c = cidx(i) + o, o in [-kk, kk]^3, with their lattice
// image n; the lanes take the atoms of each cell 32 at a time, and a ballot
// keeps the hits in cell order, then atom order.  FILL = false counts, FILL =
// true writes (j, packed n) for the pairs below cap.  The order is fixed, so
// the list is the same on every run.  err bit 1: an image index beyond +-127.
template <bool FILL>
__global__ void __launch_bounds__(128) k_neighbors(NeighborGrid ng, const double *__restrict__ pos,
                                                   int *__restrict__ cnt_or_row, int *__restrict__ col,
                                                   int *__restrict__ shift, int *__restrict__ err, long long cap) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (i >= ng.N) return;
    const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    int c = 0;
    const int base = FILL ? cnt_or_row[i] : 0;
    for (int o0 = -ng.kk[0]; o0 <= ng.kk[0]; ++o0) {
        const int t0 = ng.cidx[3 * i] + o0;
        const int n0 = t0 >= 0 ? t0 / ng.nc[0] : -((-t0 + ng.nc[0] - 1) / ng.nc[0]);
        const int b0 = t0 - n0 * ng.nc[0];
        for (int o1 = -ng.kk[1]; o1 <= ng.kk[1]; ++o1) {
            const int t1 = ng.cidx[3 * i + 1] + o1;
            const int n1 = t1 >= 0 ? t1 / ng.nc[1] : -((-t1 + ng.nc[1] - 1) / ng.nc[1]);
            const int b1 = t1 - n1 * ng.nc[1];
            for (int o2 = -ng.kk[2]; o2 <= ng.kk[2]; ++o2) {
                const int t2 = ng.cidx[3 * i + 2] + o2;
                const int n2 = t2 >= 0 ? t2 / ng.nc[2] : -((-t2 + ng.nc[2] - 1) / ng.nc[2]);
                const int b2 = t2 - n2 * ng.nc[2];
                const int cell = (b0 * ng.nc[1] + b1) * ng.nc[2] + b2;
                const double sx = n0 * ng.cell[0] + n1 * ng.cell[3] + n2 * ng.cell[6];
                const double sy = n0 * ng.cell[1] + n1 * ng.cell[4] + n2 * ng.cell[7];
                const double sz = n0 * ng.cell[2] + n1 * ng.cell[5] + n2 * ng.cell[8];
                const bool far = abs(n0) > 127 || abs(n1) > 127 || abs(n2) > 127;
                const int q0 = ng.start[cell], q1 = ng.start[cell + 1];
                for (int qb = q0; qb < q1; qb += 32) {
                    const int q = qb + lane;
                    bool hit = false;
                    int j = 0;
                    if (q < q1) {
                        j = ng.atoms[q];
                        const double rx = px - pos[3 * j] - sx, ry = py - pos[3 * j + 1] - sy,
                                     rz = pz - pos[3 * j + 2] - sz;
                        const double r2 = rx * rx + ry * ry + rz * rz;
                        hit = r2 < ng.r2max && r2 > 0.0;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, hit);
                    if (hit && far && !FILL) atomicOr(err, 1);
                    if (FILL && hit && !far) {
                        const int at = base + c + __popc(bal & ((1u << lane) - 1u));
                        if (at < cap) {
                            col[at] = j;
                            shift[at] = (n0 + 128) | ((n1 + 128) << 8) | ((n2 + 128) << 16);
                        }
                    }
                    c += __popc(bal);
                }
            }
        }
    }
    if (!FILL && lane == 0) cnt_or_row[i] = c;
}

template <class T> PrecData<T> &prec(mbd_system *s);
template <> PrecData<double> &prec<double>(mbd_system *s) { return s->f64; }
template <> PrecData<float> &prec<float>(mbd_system *s) { return s->f32; }

}  // namespace

template <class T> mbd_status launch_pair_tensors(mbd_system *s, cudaStream_t st) {
    PrecData<T> &P = prec<T>(s);
    const size_t cap = (size_t)std::max<long long>(1, s->nb_cap);
    MBD_TRY(P.pairA.ensure(sizeof(T) * 6 * cap));
    MBD_TRY(P.pairdA.ensure(sizeof(T) * 18 * cap));
    const Geom g = make_geom(s);
    const int threads = 256;
    const int blocks = (int)(((long long)s->N * 32 + threads - 1) / threads);
    k_pair_tensors<T><<<blocks, threads, 0, st>>>(s->N, s->pos_d.as<double>(), s->rvdw_d.as<double>(),
                                                  s->row_d.as<int>(), s->col_d.as<int>(), s->shift_d.as<int>(), g,
                                                  s->ewald_beta, s->r_cut, s->damp_cut, s->damp_beta, s->damp_d,
                                                  P.pairA.template as<T>(), P.pairdA.template as<T>(),
                                                  (long long)cap);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T> mbd_status launch_splines(mbd_system *s, cudaStream_t st) {
    PrecData<T> &P = prec<T>(s);
    const size_t n = (size_t)s->N * 3 * s->p;
    MBD_TRY(P.w.ensure(sizeof(T) * n));
    MBD_TRY(P.dw.ensure(sizeof(T) * n));
    MBD_TRY(P.d2w.ensure(sizeof(T) * n));
    MBD_TRY(s->w64_d.ensure(sizeof(double) * n));
    MBD_TRY(s->dw64_d.ensure(sizeof(double) * n));
    const Geom g = make_geom(s);
    const int threads = 256;
    k_splines<T><<<(3 * s->N + threads - 1) / threads, threads, 0, st>>>(
        s->N, s->pos_d.as<double>(), g, s->top_d.as<int>(), P.w.template as<T>(), P.dw.template as<T>(),
        P.d2w.template as<T>(), s->w64_d.as<double>(), s->dw64_d.as<double>());
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T> mbd_status launch_influence(mbd_system *s, const double *bmod_host, cudaStream_t st) {
    PrecData<T> &P = prec<T>(s);
    const size_t total = (size_t)s->K[0] * s->K[1] * s->K[2];
    MBD_TRY(P.G.ensure(sizeof(T) * total));
    DevBuf bm;
    const size_t nb = (size_t)(s->K[0] + s->K[1] + s->K[2]);
    MBD_TRY(bm.ensure(sizeof(double) * nb));
    MBD_CUDA_TRY(cudaMemcpyAsync(bm.ptr, bmod_host, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    const Geom g = make_geom(s);
    const int threads = 256;
    k_influence<T><<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(g, bm.as<double>(), s->ewald_beta,
                                                                                   s->volume, P.G.template as<T>());
    MBD_LAUNCH_CHECK();
    MBD_CUDA_TRY(cudaStreamSynchronize(st));   // bm is freed on return
    return MBD_OK;
}

mbd_status launch_neighbors(const NeighborGrid &ng, const double *pos, int *cnt_or_row, int *col, int *shift,
                            int *err, bool fill, long long cap, cudaStream_t st) {
    const unsigned blocks = (unsigned)((ng.N + 3) / 4);   // a warp per atom
    if (ng.N == 0) return MBD_OK;
    if (fill)
        k_neighbors<true><<<blocks, 128, 0, st>>>(ng, pos, cnt_or_row, col, shift, err, cap);
    else
        k_neighbors<false><<<blocks, 128, 0, st>>>(ng, pos, cnt_or_row, col, shift, err, cap);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

namespace {
// Brick of each atom (of its top stencil point) and the atoms per brick.
__global__ void k_bin_count(int N, const int *__restrict__ top, BinView B, int *__restrict__ bin_of,
                            int *__restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = (top[3 * i] / B.bs1 * B.nb2 + top[3 * i + 1] / B.bs2) * B.nb3 + top[3 * i + 2] / B.bs3;
    bin_of[i] = b;
    atomicAdd(&cnt[b], 1);
}
// Each atom takes a slot of its brick (in arrival order) ...
__global__ void k_bin_fill(int N, const int *__restrict__ bin_of, int *__restrict__ cursor, int *__restrict__ atoms) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    atoms[atomicAdd(&cursor[bin_of[i]], 1)] = i;
}
// ... and each brick's atoms are then put in increasing index order, so the
// lists do not depend on the arrival order.
__global__ void k_bin_sort(int nbins, const int *__restrict__ start, int *__restrict__ atoms) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int q0 = start[b], q1 = start[b + 1];
    for (int q = q0 + 1; q < q1; ++q) {
        const int v = atoms[q];
        int r = q - 1;
        while (r >= q0 && atoms[r] > v) {
            atoms[r + 1] = atoms[r];
            --r;
        }
        atoms[r + 1] = v;
    }
}

// ---------------------------------------------------------------- Morton order of the bricks
__device__ __forceinline__ unsigned morton_spread3(unsigned v) {   // bits b -> 3b
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ unsigned morton_compact3(unsigned v) {  // 3b -> b
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x3ffu;
    return v;
}
// cnt[m] = atoms of the brick at Morton index m of an M^3 cube (0 outside the brick grid)
__global__ void k_morton_count(unsigned mtotal, BinView B, int *__restrict__ cnt) {
    const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= mtotal) return;
    const int b1 = (int)morton_compact3(m >> 2), b2 = (int)morton_compact3(m >> 1), b3 = (int)morton_compact3(m);
    int c = 0;
    if (b1 < B.nb1 && b2 < B.nb2 && b3 < B.nb3) {
        const int bin = (b1 * B.nb2 + b2) * B.nb3 + b3;
        c = B.start[bin + 1] - B.start[bin];
    }
    cnt[m] = c;
}
__global__ void k_morton_fill(unsigned mtotal, BinView B, const int *__restrict__ start, int *__restrict__ order) {
    const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= mtotal) return;
    const int b1 = (int)morton_compact3(m >> 2), b2 = (int)morton_compact3(m >> 1), b3 = (int)morton_compact3(m);
    if (b1 >= B.nb1 || b2 >= B.nb2 || b3 >= B.nb3) return;
    const int bin = (b1 * B.nb2 + b2) * B.nb3 + b3;
    const int o = start[m];
    for (int s = B.start[bin]; s < B.start[bin + 1]; ++s) order[o + (s - B.start[bin])] = B.atoms[s];
}

// ---------------------------------------------------------------- clusters of the real-space field
// Cluster c is the atoms order[16c .. 16c + 15] (consecutive in the Morton order
// of the bricks, so close in space).  Its entries are the distinct neighbours
// j of its atoms (over all images), in increasing j; its pairs are grouped by
// the cluster atom il (pair starts per (c, il)) and, within an atom, ordered
// by (j, image), each carrying the index of its entry and its pair tensor.
// A block per cluster sorts the cluster's pairs in shared memory (bitonic,
// keys (j, image, il), il in the low 4 bits); COUNT = true counts entries and pairs, COUNT = false
// writes them at the scanned starts.
__device__ __forceinline__ void bitonic_sort_smem(unsigned long long *key, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ij = i ^ j;
                if (ij > i) {
                    const unsigned long long a = key[i], b = key[ij];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        key[i] = b;
                        key[ij] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <class T, bool COUNT>
__global__ void __launch_bounds__(256) k_cluster_pairs(int N, int nclus, const int *__restrict__ order,
                                                       const int *__restrict__ row, const int *__restrict__ col,
                                                       const int *__restrict__ shift, const double *__restrict__ pos,
                                                       const double *__restrict__ rvdw, Geom g, double beta,
                                                       double r_cut, double damp_cut, double damp_beta, double damp_d,
                                                       int *__restrict__ ecnt, int *__restrict__ pcnt,
                                                       int *__restrict__ entries, RealPair<T> *__restrict__ pairs,
                                                       int *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char cl_smem[];   // kClusterSortCap keys, entry indices, slots
    unsigned long long *key = reinterpret_cast<unsigned long long *>(cl_smem);
    int *eidx = reinterpret_cast<int *>(key + kClusterSortCap);
    int *slot = eidx + kClusterSortCap;
    __shared__ int at[kClusterSize], rb[kClusterSize + 1], ilstart[kClusterSize];
    __shared__ int s_total;
    const int c = blockIdx.x;
    if (c >= nclus) return;
    if (threadIdx.x < kClusterSize) {
        const int idx = c * kClusterSize + threadIdx.x;
        at[threadIdx.x] = idx < N ? order[idx] : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rb[0] = 0;
        for (int l = 0; l < kClusterSize; ++l) rb[l + 1] = rb[l] + (at[l] >= 0 ? row[at[l] + 1] - row[at[l]] : 0);
        s_total = rb[kClusterSize];
    }
    __syncthreads();
    const int total = s_total;
    if (total > kClusterSortCap) {                 // the caller falls back to per-atom pairs
        if (threadIdx.x == 0) {
            atomicOr(err, 1);
            if (COUNT) {
                ecnt[c] = 0;
                for (int l = 0; l < kClusterSize; ++l) pcnt[c * kClusterSize + l] = 0;
            }
        }
        return;
    }
    int n = 1;
    while (n < total) n <<= 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        unsigned long long kv = ~0ull;
        if (k < total) {
            int l = 0;
            while (rb[l + 1] <= k) ++l;
            const int q = row[at[l]] + (k - rb[l]);
            kv = ((unsigned long long)col[q] << 28) | ((unsigned long long)(shift[q] & 0xffffff) << 4) |
                 (unsigned long long)l;
        }
        key[k] = kv;
    }
    __syncthreads();
    bitonic_sort_smem(key, n);
    // entry index of every pair (a new entry at each new j) and its slot
    // among the pairs of its atom (order of the sorted keys)
    if (threadIdx.x == 0) {   // serial (at most kClusterSortCap pairs; setup only)
        int ne = 0, cnt[kClusterSize];
        for (int l = 0; l < kClusterSize; ++l) cnt[l] = 0;
        for (int k = 0; k < total; ++k) {
            if (k == 0 || (key[k] >> 28) != (key[k - 1] >> 28)) ++ne;
            eidx[k] = ne - 1;
            const int l = (int)(key[k] & 15ull);
            slot[k] = cnt[l]++;
        }
        int acc = 0;
        for (int l = 0; l < kClusterSize; ++l) {
            ilstart[l] = acc;
            acc += cnt[l];
            if (COUNT) pcnt[c * kClusterSize + l] = cnt[l];
        }
        if (COUNT) ecnt[c] = ne;
    }
    __syncthreads();
    if (COUNT) return;
    const int e0 = ecnt[c], p0 = pcnt[c * kClusterSize];   // scanned starts
    for (int k = threadIdx.x; k < total; k += blockDim.x) {
        const int il = (int)(key[k] & 15ull), j = (int)(key[k] >> 28), sh = (int)((key[k] >> 4) & 0xffffff);
        if (k == 0 || eidx[k] != eidx[k - 1]) entries[e0 + eidx[k]] = j;
        // the pair tensor of atom il and (j, image), FP64 from the positions
        const int i = at[il];
        const double n1 = double((sh & 255) - 128), n2 = double(((sh >> 8) & 255) - 128),
                     n3 = double(((sh >> 16) & 255) - 128);
        const double rx = pos[3 * i] - pos[3 * j] - (n1 * g.cell[0] + n2 * g.cell[3] + n3 * g.cell[6]);
        const double ry = pos[3 * i + 1] - pos[3 * j + 1] - (n1 * g.cell[1] + n2 * g.cell[4] + n3 * g.cell[7]);
        const double rz = pos[3 * i + 2] - pos[3 * j + 2] - (n1 * g.cell[2] + n2 * g.cell[5] + n3 * g.cell[8]);
        const PairRadial pr = pair_radial(rx * rx + ry * ry + rz * rz, rvdw[i] + rvdw[j], beta, r_cut, damp_cut,
                                          damp_beta, damp_d);
        RealPair<T> rp;
        rp.e = eidx[k];
        rp.pad = 0;
        rp.a[0] = T(pr.cid - pr.crr * rx * rx);
        rp.a[1] = T(-pr.crr * rx * ry);
        rp.a[2] = T(-pr.crr * rx * rz);
        rp.a[3] = T(pr.cid - pr.crr * ry * ry);
        rp.a[4] = T(-pr.crr * ry * rz);
        rp.a[5] = T(pr.cid - pr.crr * rz * rz);
        pairs[(size_t)p0 + ilstart[il] + slot[k]] = rp;
    }
}
}  // namespace

// Atoms in the Morton order of their bricks (bins): close atoms are close in
// the order, in compact groups.  order: [N].  Returns MBD_ERR_UNSUPPORTED when
// the brick grid is too large for the Morton cube (the caller keeps the
// brick-major order).
mbd_status launch_morton_order(const BinView &B, int N, int *order, DevBuf &cnt, DevBuf &start, DevBuf &bsum,
                               cudaStream_t st) {
    int M = 1;
    while (M < B.nb1 || M < B.nb2 || M < B.nb3) M <<= 1;
    const unsigned long long mtotal = (unsigned long long)M * M * M;
    if (mtotal > (1ull << 24) || M > 1024) return MBD_ERR_UNSUPPORTED;
    MBD_TRY(cnt.ensure(sizeof(int) * mtotal));
    MBD_TRY(start.ensure(sizeof(int) * (mtotal + 1)));
    const unsigned blocks = (unsigned)((mtotal + 255) / 256);
    k_morton_count<<<blocks, 256, 0, st>>>((unsigned)mtotal, B, cnt.as<int>());
    MBD_LAUNCH_CHECK();
    MBD_TRY(launch_exclusive_scan(cnt.as<int>(), start.as<int>(), (int)mtotal, bsum, st));
    if (N > 0) {
        k_morton_fill<<<blocks, 256, 0, st>>>((unsigned)mtotal, B, start.as<int>(), order);
        MBD_LAUNCH_CHECK();
    }
    return MBD_OK;
}

// The clusters of the real-space field (k_cluster_pairs): counts, scans of
// the entry starts (per cluster) and pair starts (per cluster atom), then
// entries and pairs.  err (device int) gets bit 1 when a cluster has more
// than kClusterSortCap pairs.
template <class T>
mbd_status launch_cluster_pairs(mbd_system *s, const int *order, int nclus, DevBuf &ecnt, DevBuf &pcnt,
                                DevBuf &estart, DevBuf &pstart, DevBuf &entries, DevBuf &A, int *err,
                                cudaStream_t st) {
    const Geom g = make_geom(s);
    const int nslots = nclus * kClusterSize;
    MBD_TRY(ecnt.ensure(sizeof(int) * std::max(1, nclus)));
    MBD_TRY(pcnt.ensure(sizeof(int) * std::max(1, nslots)));
    MBD_TRY(estart.ensure(sizeof(int) * (nclus + 1)));
    MBD_TRY(pstart.ensure(sizeof(int) * (nslots + 1)));
    const size_t cap = (size_t)std::max<long long>(1, s->nb_cap);
    MBD_TRY(entries.ensure(sizeof(int) * cap));
    MBD_TRY(A.ensure(sizeof(RealPair<T>) * cap));
    if (nclus == 0) return MBD_OK;
    const size_t smem = (size_t)kClusterSortCap * (sizeof(unsigned long long) + 2 * sizeof(int));
    MBD_CUDA_TRY(cudaFuncSetAttribute(k_cluster_pairs<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MBD_CUDA_TRY(cudaFuncSetAttribute(k_cluster_pairs<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_cluster_pairs<T, true><<<nclus, 256, smem, st>>>(
        s->N, nclus, order, s->row_d.as<int>(), s->col_d.as<int>(), s->shift_d.as<int>(), s->pos_d.as<double>(),
        s->rvdw_d.as<double>(), g, s->ewald_beta, s->r_cut, s->damp_cut, s->damp_beta, s->damp_d, ecnt.as<int>(),
        pcnt.as<int>(), nullptr, (RealPair<T> *)nullptr, err);
    MBD_LAUNCH_CHECK();
    MBD_TRY(launch_exclusive_scan(ecnt.as<int>(), estart.as<int>(), nclus, s->scan_bsum, st));
    MBD_TRY(launch_exclusive_scan(pcnt.as<int>(), pstart.as<int>(), nslots, s->scan_bsum, st));
    k_cluster_pairs<T, false><<<nclus, 256, smem, st>>>(
        s->N, nclus, order, s->row_d.as<int>(), s->col_d.as<int>(), s->shift_d.as<int>(), s->pos_d.as<double>(),
        s->rvdw_d.as<double>(), g, s->ewald_beta, s->r_cut, s->damp_cut, s->damp_beta, s->damp_d,
        estart.as<int>(), pstart.as<int>(), entries.as<int>(), A.template as<RealPair<T>>(), err);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}
template mbd_status launch_cluster_pairs<double>(mbd_system *, const int *, int, DevBuf &, DevBuf &, DevBuf &,
                                                 DevBuf &, DevBuf &, DevBuf &, int *, cudaStream_t);
template mbd_status launch_cluster_pairs<float>(mbd_system *, const int *, int, DevBuf &, DevBuf &, DevBuf &,
                                                DevBuf &, DevBuf &, DevBuf &, int *, cudaStream_t);

mbd_status launch_bin_atoms(int N, const int *top, const BinView &B, int *bin_of, int *cnt, int *start,
                            int *cursor, int *atoms, DevBuf &bsum, cudaStream_t st) {
    const int nbins = B.nb1 * B.nb2 * B.nb3;
    MBD_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * nbins, st));
    if (N > 0) {
        k_bin_count<<<(N + 255) / 256, 256, 0, st>>>(N, top, B, bin_of, cnt);
        MBD_LAUNCH_CHECK();
    }
    MBD_TRY(launch_exclusive_scan(cnt, start, nbins, bsum, st));
    MBD_CUDA_TRY(cudaMemcpyAsync(cursor, start, sizeof(int) * nbins, cudaMemcpyDeviceToDevice, st));
    if (N > 0) {
        k_bin_fill<<<(N + 255) / 256, 256, 0, st>>>(N, bin_of, cursor, atoms);
        MBD_LAUNCH_CHECK();
        k_bin_sort<<<(nbins + 255) / 256, 256, 0, st>>>(nbins, start, atoms);
        MBD_LAUNCH_CHECK();
    }
    return MBD_OK;
}

template mbd_status launch_pair_tensors<double>(mbd_system *, cudaStream_t);
template mbd_status launch_pair_tensors<float>(mbd_system *, cudaStream_t);
template mbd_status launch_splines<double>(mbd_system *, cudaStream_t);
template mbd_status launch_splines<float>(mbd_system *, cudaStream_t);
template mbd_status launch_influence<double>(mbd_system *, const double *, cudaStream_t);
template mbd_status launch_influence<float>(mbd_system *, const double *, cudaStream_t);

}  // namespace mbd
