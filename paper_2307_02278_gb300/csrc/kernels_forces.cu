// Force kernels.  The paper computes energies only (its Conclusions name the
// gradients as the next step); with alpha and omega position-independent,
//   dE/dR = (1/4) Tr(C^{-1/2} dC/dR) ~ (1/4)(D/R) sum_l grad_R [p_l^T T'(R) q_l],
// p_l = g . w_l, q_l = g . v_l, w_l = C^{-1/2} v_l = sum_k c_{lk} y_{lk}.
// The probes' p and q are interleaved as one complex probe pair, so the SPME
// part reuses the spread and FFT convolution kernels with 2R "probes":
//   phi_p + i phi_q = F^-1[G F[D_p + i D_q]],
// and grad_i = sum_k H_i(k) [p_i phi_q(k) + q_i phi_p(k)] with H_i the Hessian
// of the stencil weight W_i(k) wrt R_i; the real-space part contracts the
// derivative of the pair tensor, dA_ab/dr_c, with p_i q_j + p_j q_i.
#include "mbd_internal.cuh"

namespace mbd {

namespace {

constexpr int kWarps = 8;

template <class T>
__global__ void k_force_dipoles(int rows, const double *__restrict__ Y, const double *__restrict__ coef,
                                const int *__restrict__ length, const double *__restrict__ g, int R, int ld, int m,
                                T *__restrict__ dpq, int ld2) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * R) return;
    const int row = (int)(idx / R), r = (int)(idx % R);
    const size_t stride = (size_t)rows * ld;
    const int n = length[r];
    double w = 0.0;
    for (int k = 0; k < n; ++k) w += coef[(size_t)k * ld + r] * Y[(size_t)k * stride + (size_t)row * ld + r];
    const double gi = g[row / 3];
    dpq[(size_t)row * ld2 + 2 * r] = T(gi * w);
    dpq[(size_t)row * ld2 + 2 * r + 1] = T(gi * Y[(size_t)row * ld + r]);
}

// The same from w = sum_k c_k y_k accumulated during a rerun of the recurrence
// (recomputed basis) and y_0 = v.
template <class T>
__global__ void k_force_dipoles_w(int rows, const double *__restrict__ w, const double *__restrict__ v,
                                  const double *__restrict__ g, int R, int ld, T *__restrict__ dpq, int ld2) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)rows * R) return;
    const int row = (int)(idx / R), r = (int)(idx % R);
    const double gi = g[row / 3];
    dpq[(size_t)row * ld2 + 2 * r] = T(gi * w[(size_t)row * ld + r]);
    dpq[(size_t)row * ld2 + 2 * r + 1] = T(gi * v[(size_t)row * ld + r]);
}

template <class T> struct ForceArgs {
    const T *dpq;        // [N][3][ld2] (p_l, q_l) interleaved
    const T *mesh;       // [K^3][ld2] (phi_p, phi_q) interleaved
    int R, ld2;
    Geom g;
    const int *top;
    const T *w, *dw, *d2w;
    const int *row, *col;
    const T *dA;         // [nnz][18] dA_ab/dr_c of the real-space pair tensor
    double scale;
    double *forces;      // [N][3] FP64
};

// WPA warps per atom: they share out the stencil planes t1 and the
// neighbours, and their partial gradients are summed in warp order.
template <class T, int WPA>
__global__ void __launch_bounds__(kWarps * 32) k_force_gather(ForceArgs<T> a) {
    static_assert(kWarps % WPA == 0, "whole atoms per block");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * (kWarps / WPA) + warp / WPA, sub = warp % WPA;
    const bool valid = i < a.g.N;
    __shared__ double part[kWarps][3];
    double gx = 0.0, gy = 0.0, gz = 0.0;
    if (valid) {
    const int p = a.g.p;
    const double *cm = a.g.cmat;
    // ---- SPME: acc_beta = sum_k sum_l H_u(k)_{beta gamma} (e_p,gamma phi_q + e_q,gamma phi_p)
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
    {
        const int top1 = a.top[3 * i], top2 = a.top[3 * i + 1], top3 = a.top[3 * i + 2];
        const T *w = a.w + (size_t)3 * p * i, *dw = a.dw + (size_t)3 * p * i, *d2w = a.d2w + (size_t)3 * p * i;
        for (int l = lane; l < a.R; l += 32) {
            // scaled-fractional components e = C x of p_i and q_i
            T pc[3], qc[3];
            for (int c = 0; c < 3; ++c) {
                pc[c] = a.dpq[(size_t)(3 * i + c) * a.ld2 + 2 * l];
                qc[c] = a.dpq[(size_t)(3 * i + c) * a.ld2 + 2 * l + 1];
            }
            T ep[3], eq[3];
            for (int b = 0; b < 3; ++b) {
                ep[b] = T(cm[3 * b]) * pc[0] + T(cm[3 * b + 1]) * pc[1] + T(cm[3 * b + 2]) * pc[2];
                eq[b] = T(cm[3 * b]) * qc[0] + T(cm[3 * b + 1]) * qc[1] + T(cm[3 * b + 2]) * qc[2];
            }
            T h0 = T(0), h1 = T(0), h2 = T(0);
            for (int t1 = sub; t1 < p; t1 += WPA) {
                int k1 = top1 - t1;
                if (k1 < 0) k1 += a.g.K1;
                const T wa = w[t1], da = dw[t1], ea = d2w[t1];
                for (int t2 = 0; t2 < p; ++t2) {
                    int k2 = top2 - t2;
                    if (k2 < 0) k2 += a.g.K2;
                    const T wb = w[p + t2], db = dw[p + t2], eb = d2w[p + t2];
                    const size_t rowbase = ((size_t)k1 * a.g.K2 + k2) * a.g.K3;
                    for (int t3 = 0; t3 < p; ++t3) {
                        int k3 = top3 - t3;
                        if (k3 < 0) k3 += a.g.K3;
                        const T wc = w[2 * p + t3], dc = dw[2 * p + t3], ec = d2w[2 * p + t3];
                        const size_t o = (rowbase + k3) * a.ld2 + 2 * l;
                        const T fp = a.mesh[o], fq = a.mesh[o + 1];
                        const T u0 = ep[0] * fq + eq[0] * fp;
                        const T u1 = ep[1] * fq + eq[1] * fp;
                        const T u2 = ep[2] * fq + eq[2] * fp;
                        const T H00 = ea * wb * wc, H11 = wa * eb * wc, H22 = wa * wb * ec;
                        const T H01 = da * db * wc, H02 = da * wb * dc, H12 = wa * db * dc;
                        h0 += H00 * u0 + H01 * u1 + H02 * u2;
                        h1 += H01 * u0 + H11 * u1 + H12 * u2;
                        h2 += H02 * u0 + H12 * u1 + H22 * u2;
                    }
                }
            }
            acc0 += double(h0);
            acc1 += double(h1);
            acc2 += double(h2);
        }
    }
    // Cartesian: grad_alpha = sum_beta C_{beta alpha} acc_beta
    gx = cm[0] * acc0 + cm[3] * acc1 + cm[6] * acc2;
    gy = cm[1] * acc0 + cm[4] * acc1 + cm[7] * acc2;
    gz = cm[2] * acc0 + cm[5] * acc1 + cm[8] * acc2;
    // ---- real space: sum_j dA_ab/dr_c sum_l (p_ia q_jb + p_ja q_ib), dA precomputed per pair
    {
        T g0 = T(0), g1 = T(0), g2 = T(0);
        for (int nb = a.row[i] + sub; nb < a.row[i + 1]; nb += WPA) {
            const int j = a.col[nb];
            T M[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
            for (int l = lane; l < a.R; l += 32) {
                T pi_[3], qi_[3], pj_[3], qj_[3];
                for (int c = 0; c < 3; ++c) {
                    pi_[c] = a.dpq[(size_t)(3 * i + c) * a.ld2 + 2 * l];
                    qi_[c] = a.dpq[(size_t)(3 * i + c) * a.ld2 + 2 * l + 1];
                    pj_[c] = a.dpq[(size_t)(3 * j + c) * a.ld2 + 2 * l];
                    qj_[c] = a.dpq[(size_t)(3 * j + c) * a.ld2 + 2 * l + 1];
                }
                int o = 0;
                for (int x = 0; x < 3; ++x)
                    for (int y = x; y < 3; ++y) {
                        T v = pi_[x] * qj_[y] + pj_[x] * qi_[y];
                        if (x != y) v += pi_[y] * qj_[x] + pj_[y] * qi_[x];
                        M[o++] += v;
                    }
            }
            const T *dA = a.dA + 18 * (size_t)nb;
            for (int ab = 0; ab < 6; ++ab) {
                g0 += dA[3 * ab] * M[ab];
                g1 += dA[3 * ab + 1] * M[ab];
                g2 += dA[3 * ab + 2] * M[ab];
            }
        }
        gx += double(g0);
        gy += double(g1);
        gz += double(g2);
    }
    }
    for (int off = 16; off > 0; off >>= 1) {
        gx += __shfl_down_sync(0xffffffffu, gx, off);
        gy += __shfl_down_sync(0xffffffffu, gy, off);
        gz += __shfl_down_sync(0xffffffffu, gz, off);
    }
    if (WPA == 1) {
        if (valid && lane == 0) {
            a.forces[3 * i] = -a.scale * gx;
            a.forces[3 * i + 1] = -a.scale * gy;
            a.forces[3 * i + 2] = -a.scale * gz;
        }
        return;
    }
    if (lane == 0) {
        part[warp][0] = gx;
        part[warp][1] = gy;
        part[warp][2] = gz;
    }
    __syncthreads();
    if (valid && sub == 0 && lane < 3) {
        double t = 0.0;
        for (int w = 0; w < WPA; ++w) t += part[warp + w][lane];
        a.forces[3 * i + lane] = -a.scale * t;
    }
}

template <class T> PrecData<T> &prec(mbd_system *s);
template <> PrecData<double> &prec<double>(mbd_system *s) { return s->f64; }
template <> PrecData<float> &prec<float>(mbd_system *s) { return s->f32; }

}  // namespace

template <class T>
mbd_status launch_force_dipoles_t(mbd_system *s, const double *Y, const double *coef, const int *length, int R,
                                  int ld, int m, T *dpq, int ld2) {
    const int rows = 3 * s->N;
    const size_t n = (size_t)rows * R;
    k_force_dipoles<T><<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(rows, Y, coef, length, s->g_d.as<double>(),
                                                                          R, ld, m, dpq, ld2);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T>
mbd_status launch_force_dipoles_w_t(mbd_system *s, const double *w, const double *v, int R, int ld, T *dpq,
                                    int ld2) {
    const int rows = 3 * s->N;
    const size_t n = (size_t)rows * R;
    k_force_dipoles_w<T><<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(rows, w, v, s->g_d.as<double>(), R,
                                                                            ld, dpq, ld2);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T>
mbd_status launch_force_gather_t(mbd_system *s, const T *dpq, const T *mesh, int R, int ld2, double scale,
                                 double *forces) {
    PrecData<T> &P = prec<T>(s);
    ForceArgs<T> a;
    a.dpq = dpq;
    a.mesh = mesh;
    a.R = R;
    a.ld2 = ld2;
    a.g.N = s->N;
    a.g.K1 = s->K[0];
    a.g.K2 = s->K[1];
    a.g.K3 = s->K[2];
    a.g.p = s->p;
    for (int b = 0; b < 3; ++b)
        for (int c = 0; c < 3; ++c) a.g.cmat[3 * b + c] = s->K[b] * s->recip[3 * b + c];
    for (int k = 0; k < 9; ++k) a.g.cell[k] = s->cell[k];
    a.top = s->top_d.as<int>();
    a.w = P.w.template as<T>();
    a.dw = P.dw.template as<T>();
    a.d2w = P.d2w.template as<T>();
    a.row = s->row_d.as<int>();
    a.col = s->col_d.as<int>();
    a.dA = P.pairdA.template as<T>();
    a.scale = scale;
    a.forces = forces;
    // warps per atom: more for small systems, whose one warp per atom would
    // leave most of the SMs' warp slots empty (3000 atoms: 272 -> 234 us with 4;
    // 24000 atoms: 2606 -> 2548 us with 2)
    const int wpa = s->N <= 8192 ? 4 : (s->N <= 65536 ? 2 : 1);
    if (wpa == 2)
        k_force_gather<T, 2><<<(s->N + kWarps / 2 - 1) / (kWarps / 2), kWarps * 32, 0, s->stream>>>(a);
    else if (wpa == 4)
        k_force_gather<T, 4><<<(s->N + kWarps / 4 - 1) / (kWarps / 4), kWarps * 32, 0, s->stream>>>(a);
    else
        k_force_gather<T, 1><<<(s->N + kWarps - 1) / kWarps, kWarps * 32, 0, s->stream>>>(a);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template mbd_status launch_force_dipoles_t<double>(mbd_system *, const double *, const double *, const int *, int, int,
                                                   int, double *, int);
template mbd_status launch_force_dipoles_t<float>(mbd_system *, const double *, const double *, const int *, int, int,
                                                  int, float *, int);
template mbd_status launch_force_dipoles_w_t<double>(mbd_system *, const double *, const double *, int, int,
                                                     double *, int);
template mbd_status launch_force_dipoles_w_t<float>(mbd_system *, const double *, const double *, int, int, float *,
                                                    int);
template mbd_status launch_force_gather_t<double>(mbd_system *, const double *, const double *, int, int, double,
                                                  double *);
template mbd_status launch_force_gather_t<float>(mbd_system *, const float *, const float *, int, int, double,
                                                 double *);

}  // namespace mbd
