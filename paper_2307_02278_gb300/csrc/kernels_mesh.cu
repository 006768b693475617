// Per-step operator kernels: SPME spreading (Eq. dipolarr), the batched 3D FFT
// convolution with the influence function (Eq. spme), and the fused field
// kernel (SPME gather + real-space pairs + self term, Eqs. spme, fld_ewald,
// fld_ewald1) with the Lanczos epilogue l_k = Omega y_k + Diag(g) E*_k and
// a_k = y_k^T l_k (Eqs. lk3, recurs2).
#include "mbd_internal.cuh"

namespace mbd {

namespace {

constexpr int kWarps = 8;          // warps per block in spread / field
constexpr int kMaxPts = 16;        // mesh points per warp in one brick (brick <= 5x5x5)

template <class T> struct SpreadArgs {
    const T *d;          // [N][3][ld] Cartesian dipoles
    T *mesh;             // [K^3][ld]
    int R, ld;
    Geom g;
    SplineView<T> sp;
    BinView bins;
};

// Deterministic spreading: one block owns one brick of mesh points and a chunk
// of 32 probes (lane = probe); it visits every atom whose stencil can reach the
// brick, in a fixed order, and writes each mesh point exactly once.  The
// Cartesian dipole is first mapped to scaled-fractional components
// e_beta = sum_alpha C_{beta alpha} d_alpha, so that
//   D(k) += e_1 M'(t1) M(t2) M(t3) + e_2 M(t1) M'(t2) M(t3) + e_3 M(t1) M(t2) M'(t3).
template <class T>
__global__ void __launch_bounds__(kWarps * 32) k_spread(SpreadArgs<T> a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < a.R;
    const BinView &B = a.bins;
    const int bidx = blockIdx.x;
    const int bb3 = bidx % B.nb3, bb2 = (bidx / B.nb3) % B.nb2, bb1 = bidx / (B.nb3 * B.nb2);
    const int o1 = bb1 * B.bs1, o2 = bb2 * B.bs2, o3 = bb3 * B.bs3;
    const int P = B.bs1 * B.bs2 * B.bs3;
    const int p = a.g.p;
    int g1[kMaxPts], g2[kMaxPts], g3[kMaxPts];
    T acc[kMaxPts];
#pragma unroll
    for (int q = 0; q < kMaxPts; ++q) {
        const int pt = warp + kWarps * q;
        acc[q] = T(0);
        const int l3 = pt % B.bs3, l2 = (pt / B.bs3) % B.bs2, l1 = pt / (B.bs3 * B.bs2);
        g1[q] = o1 + l1;
        g2[q] = o2 + l2;
        g3[q] = o3 + l3;
    }
    const T c00 = T(a.g.cmat[0]), c01 = T(a.g.cmat[1]), c02 = T(a.g.cmat[2]);
    const T c10 = T(a.g.cmat[3]), c11 = T(a.g.cmat[4]), c12 = T(a.g.cmat[5]);
    const T c20 = T(a.g.cmat[6]), c21 = T(a.g.cmat[7]), c22 = T(a.g.cmat[8]);
    for (int c1 = 0; c1 < B.nc1; ++c1) {
        const int t1 = (bb1 + c1) % B.nb1;
        for (int c2 = 0; c2 < B.nc2; ++c2) {
            const int t2 = (bb2 + c2) % B.nb2;
            for (int c3 = 0; c3 < B.nc3; ++c3) {
                const int t3 = (bb3 + c3) % B.nb3;
                const int bin = (t1 * B.nb2 + t2) * B.nb3 + t3;
                const int s0 = B.start[bin], s1 = B.start[bin + 1];
                for (int s = s0; s < s1; ++s) {
                    const int j = B.atoms[s];
                    T d0 = T(0), d1 = T(0), d2 = T(0);
                    if (valid) {
                        d0 = a.d[(size_t)(3 * j) * a.ld + r];
                        d1 = a.d[(size_t)(3 * j + 1) * a.ld + r];
                        d2 = a.d[(size_t)(3 * j + 2) * a.ld + r];
                    }
                    const T e0 = c00 * d0 + c01 * d1 + c02 * d2;
                    const T e1 = c10 * d0 + c11 * d1 + c12 * d2;
                    const T e2 = c20 * d0 + c21 * d1 + c22 * d2;
                    const int top1 = a.sp.top[3 * j], top2 = a.sp.top[3 * j + 1], top3 = a.sp.top[3 * j + 2];
                    const T *w = a.sp.w + (size_t)3 * p * j;
                    const T *dw = a.sp.dw + (size_t)3 * p * j;
#pragma unroll
                    for (int q = 0; q < kMaxPts; ++q) {
                        if (warp + kWarps * q >= P) break;
                        int u1 = top1 - g1[q];
                        if (u1 < 0) u1 += a.g.K1;
                        if (u1 >= p) continue;
                        int u2 = top2 - g2[q];
                        if (u2 < 0) u2 += a.g.K2;
                        if (u2 >= p) continue;
                        int u3 = top3 - g3[q];
                        if (u3 < 0) u3 += a.g.K3;
                        if (u3 >= p) continue;
                        const T m1 = w[u1], m2 = w[p + u2], m3 = w[2 * p + u3];
                        const T n1 = dw[u1], n2 = dw[p + u2], n3 = dw[2 * p + u3];
                        acc[q] += e0 * (n1 * m2 * m3) + e1 * (m1 * n2 * m3) + e2 * (m1 * m2 * n3);
                    }
                }
            }
        }
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < kMaxPts; ++q) {
        if (warp + kWarps * q >= P) break;
        const size_t pt = ((size_t)g1[q] * a.g.K2 + g2[q]) * a.g.K3 + g3[q];
        a.mesh[pt * a.ld + r] = acc[q];
    }
}

// ---------------------------------------------------------------- FFT
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
// multiply by -i*sign... rot(a) = sign * i * a, with sign = -1 (forward) or +1 (inverse)
template <class C> __device__ __forceinline__ C rot(C a, int sign) {
    return sign < 0 ? C{a.y, -a.x} : C{-a.y, a.x};
}

// In-register R-point DFT  X_t = sum_q x_q exp(sign 2 pi i q t / R), R in {2,3,4,5,8}.
template <class T, class C> __device__ __forceinline__ void dft2(C *v) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <class T, class C> __device__ __forceinline__ void dft4(C *v, int sign) {
    const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const C s13 = cadd(v[1], v[3]), d13 = rot(csub(v[1], v[3]), sign);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
template <class T, class C> __device__ __forceinline__ void dft8(C *v, int sign) {
    const T h = T(0.70710678118654752440);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T>(e, sign);
    dft4<T>(o, sign);
    // twiddles exp(sign 2 pi i t / 8), t = 0..3
    const C o1 = C{h * (o[1].x - T(sign) * o[1].y), h * (o[1].y + T(sign) * o[1].x)};
    const C o2 = rot(o[2], sign);
    const C o3 = C{h * (-o[3].x - T(sign) * o[3].y), h * (-o[3].y + T(sign) * o[3].x)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
}
template <class T, class C> __device__ __forceinline__ void dft3(C *v, int sign) {
    const T c = T(-0.5), s = T(sign) * T(0.86602540378443864676);
    const C a = v[0], b = v[1], d = v[2];
    const C t = cadd(b, d);
    const C u = csub(b, d);
    v[0] = cadd(a, t);
    const C m = C{a.x + c * t.x, a.y + c * t.y};
    const C n = C{-s * u.y, s * u.x};   // i s (b - d)
    v[1] = cadd(m, n);
    v[2] = csub(m, n);
}
template <class T, class C> __device__ __forceinline__ void dft5(C *v, int sign) {
    // cos/sin of 2 pi / 5 and 4 pi / 5
    const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
    const T s1 = T(sign) * T(0.95105651629515357212), s2 = T(sign) * T(0.58778525229247312917);
    const C a = v[0];
    const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const C u1 = csub(v[1], v[4]), u2 = csub(v[2], v[3]);
    v[0] = C{a.x + t1.x + t2.x, a.y + t1.y + t2.y};
    const C m1 = C{a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
    const C m2 = C{a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
    // i (s1 u1 + s2 u2) and i (s2 u1 - s1 u2)
    const C n1 = C{-(s1 * u1.y + s2 * u2.y), s1 * u1.x + s2 * u2.x};
    const C n2 = C{-(s2 * u1.y - s1 * u2.y), s2 * u1.x - s1 * u2.x};
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
}

template <class T> struct FFTArgs {
    typename Cplx<T>::type *data;   // complex view of the mesh
    const typename Cplx<T>::type *tw;   // exp(-2 pi i n / K), n = 0..K-1
    const T *G;          // influence function (fused pass only)
    int K;
    int inner;           // complex elements per row (contiguous)
    int W;               // tile width (complex columns)
    int nst;
    int radix[kMaxRadixStages];
    int V;               // complex probe pairs per mesh point (fused pass: G index = e / V)
    int sign;            // -1 forward, +1 inverse (unfused passes)
};

// Mixed-radix Stockham passes over the K rows of a K x W tile held in shared
// memory; returns the buffer that holds the result (natural order).
template <class T, class C>
__device__ C *stockham(C *in, C *out, const FFTArgs<T> &a, int sign) {
    const int K = a.K, W = a.W;
    int Ns = 1;
    for (int s = 0; s < a.nst; ++s) {
        const int R = a.radix[s];
        const int nb = K / R;
        const int step = K / (Ns * R);
        for (int idx = threadIdx.x; idx < nb * W; idx += blockDim.x) {
            const int j = idx / W, col = idx - j * W;
            C v[8];
            for (int q = 0; q < R; ++q) v[q] = in[(j + q * nb) * W + col];
            const int jm = j % Ns;
            if (jm != 0) {
                for (int q = 1; q < R; ++q) {
                    C t = a.tw[q * jm * step];
                    if (sign > 0) t.y = -t.y;
                    v[q] = cmul(v[q], t);
                }
            }
            switch (R) {
                case 2: dft2<T>(v); break;
                case 3: dft3<T>(v, sign); break;
                case 4: dft4<T>(v, sign); break;
                case 5: dft5<T>(v, sign); break;
                default: dft8<T>(v, sign); break;
            }
            const int base = (j / Ns) * Ns * R + jm;
            for (int q = 0; q < R; ++q) out[(base + q * Ns) * W + col] = v[q];
        }
        __syncthreads();
        C *t = in;
        in = out;
        out = t;
        Ns *= R;
    }
    return in;
}

// One 1D FFT pass along the middle axis of [outer][K][inner] (complex); with
// FUSED the pass is forward, then multiplies by G(k1, k2, k3), then inverse.
template <class T, bool FUSED>
__global__ void __launch_bounds__(256) k_fft_pass(FFTArgs<T> a) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *b0 = reinterpret_cast<C *>(smem_raw);
    C *b1 = b0 + a.K * a.W;
    const int ncb = (a.inner + a.W - 1) / a.W;
    const size_t outer = blockIdx.x / ncb;
    const int c0 = (int)(blockIdx.x % ncb) * a.W;
    const int wc = min(a.W, a.inner - c0);
    C *base = a.data + outer * (size_t)a.K * a.inner + c0;
    for (int idx = threadIdx.x; idx < a.K * a.W; idx += blockDim.x) {
        const int row = idx / a.W, col = idx - row * a.W;
        b0[idx] = col < wc ? base[(size_t)row * a.inner + col] : C{T(0), T(0)};
    }
    __syncthreads();
    C *res;
    if (FUSED) {
        res = stockham<T, C>(b0, b1, a, -1);
        C *other = (res == b0) ? b1 : b0;
        // G index: k1 = row, (k2, k3) = (c0 + col) / V
        for (int idx = threadIdx.x; idx < a.K * a.W; idx += blockDim.x) {
            const int row = idx / a.W, col = idx - row * a.W;
            if (col < wc) {
                const T gv = a.G[(size_t)row * (a.inner / a.V) + (c0 + col) / a.V];
                res[idx].x *= gv;
                res[idx].y *= gv;
            }
        }
        __syncthreads();
        res = stockham<T, C>(res, other, a, +1);
    } else {
        res = stockham<T, C>(b0, b1, a, a.sign);
    }
    for (int idx = threadIdx.x; idx < a.K * a.W; idx += blockDim.x) {
        const int row = idx / a.W, col = idx - row * a.W;
        if (col < wc) base[(size_t)row * a.inner + col] = res[idx];
    }
}

// ---------------------------------------------------------------- field
template <class T> struct FieldArgs {
    const T *d;          // [N][3][ld]
    const T *mesh;       // [K^3][ld]
    int R, ld;
    Geom g;
    SplineView<T> sp;
    PairView<T> pr;
    const int *order;    // atom processing order (spatially sorted)
    const double *g_at;  // [N] w sqrt(alpha)
    const double *w2;    // [N] w^2
    double self_coef;
    FieldOut<T> o;
};

// One warp per atom, lane = probe.  E* = E^rec + E^dir + E^self, then the
// epilogue selected by o.mode.
template <class T>
__global__ void __launch_bounds__(kWarps * 32) k_field(FieldArgs<T> a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y * 32 + lane;
    const bool valid = r < a.R;
    const int idx = blockIdx.x * kWarps + warp;
    const int p = a.g.p;
    double part = 0.0;
    if (idx < a.g.N) {
        const int i = a.order[idx];
        T E0 = T(0), E1 = T(0), E2 = T(0);
        if (a.o.terms & MBD_TERM_RECIP) {
            T f0 = T(0), f1 = T(0), f2 = T(0);
            const int top1 = a.sp.top[3 * i], top2 = a.sp.top[3 * i + 1], top3 = a.sp.top[3 * i + 2];
            const T *w = a.sp.w + (size_t)3 * p * i;
            const T *dw = a.sp.dw + (size_t)3 * p * i;
            for (int t1 = 0; t1 < p; ++t1) {
                int k1 = top1 - t1;
                if (k1 < 0) k1 += a.g.K1;
                const T wa = w[t1], da = dw[t1];
                for (int t2 = 0; t2 < p; ++t2) {
                    int k2 = top2 - t2;
                    if (k2 < 0) k2 += a.g.K2;
                    const T wb = w[p + t2], db = dw[p + t2];
                    const T ab = wa * wb, Ab = da * wb, aB = wa * db;
                    const size_t rowbase = ((size_t)k1 * a.g.K2 + k2) * a.g.K3;
                    for (int t3 = 0; t3 < p; ++t3) {
                        int k3 = top3 - t3;
                        if (k3 < 0) k3 += a.g.K3;
                        const T wc = w[2 * p + t3], dc = dw[2 * p + t3];
                        const T phi = valid ? a.mesh[(rowbase + k3) * a.ld + r] : T(0);
                        f0 += (Ab * wc) * phi;
                        f1 += (aB * wc) * phi;
                        f2 += (ab * dc) * phi;
                    }
                }
            }
            // E^rec_alpha = sum_beta C_{beta alpha} f_beta
            E0 += T(a.g.cmat[0]) * f0 + T(a.g.cmat[3]) * f1 + T(a.g.cmat[6]) * f2;
            E1 += T(a.g.cmat[1]) * f0 + T(a.g.cmat[4]) * f1 + T(a.g.cmat[7]) * f2;
            E2 += T(a.g.cmat[2]) * f0 + T(a.g.cmat[5]) * f1 + T(a.g.cmat[8]) * f2;
        }
        if (a.o.terms & MBD_TERM_REAL) {
            const int nb0 = a.pr.row[i], nb1 = a.pr.row[i + 1];
            for (int nb = nb0; nb < nb1; ++nb) {
                const int j = a.pr.col[nb];
                const T *A = a.pr.A + 6 * (size_t)nb;
                const T A0 = A[0], A1 = A[1], A2 = A[2], A3 = A[3], A4 = A[4], A5 = A[5];
                T x = T(0), y = T(0), z = T(0);
                if (valid) {
                    x = a.d[(size_t)(3 * j) * a.ld + r];
                    y = a.d[(size_t)(3 * j + 1) * a.ld + r];
                    z = a.d[(size_t)(3 * j + 2) * a.ld + r];
                }
                E0 += A0 * x + A1 * y + A2 * z;
                E1 += A1 * x + A3 * y + A4 * z;
                E2 += A2 * x + A4 * y + A5 * z;
            }
        }
        if ((a.o.terms & MBD_TERM_SELF) && valid) {
            const T c = T(a.self_coef);
            E0 += c * a.d[(size_t)(3 * i) * a.ld + r];
            E1 += c * a.d[(size_t)(3 * i + 1) * a.ld + r];
            E2 += c * a.d[(size_t)(3 * i + 2) * a.ld + r];
        }
        if (valid) {
            const double E[3] = {double(E0), double(E1), double(E2)};
            const size_t rows[3] = {(size_t)(3 * i) * a.ld + r, (size_t)(3 * i + 1) * a.ld + r,
                                    (size_t)(3 * i + 2) * a.ld + r};
            if (a.o.mode == kFieldOut) {
                for (int c = 0; c < 3; ++c) a.o.out[rows[c]] = E[c];
            } else if (a.o.mode == kFieldApply) {
                const double w2 = a.w2[i], gi = a.g_at[i];
                for (int c = 0; c < 3; ++c) a.o.out[rows[c]] = w2 * a.o.xin[rows[c]] + gi * E[c];
            } else {
                const double invb = a.o.lz.invb[r];
                const double w2 = a.w2[i], gi = a.g_at[i];
                double *Yk = a.o.lz.Y + (size_t)a.o.k * (size_t)(3 * a.g.N) * a.ld;
                for (int c = 0; c < 3; ++c) {
                    const double y = Yk[rows[c]] * invb;
                    const double l = w2 * y + gi * E[c] * invb;
                    Yk[rows[c]] = y;
                    a.o.lz.L[rows[c]] = l;
                    part += y * l;
                }
            }
        }
    }
    if (a.o.mode != kFieldLanczos) return;
    // a_k = y_k^T l_k: block partial per probe, then the last block sums the
    // partials in block order (deterministic) and resets the counter.
    __shared__ double red[kWarps][32];
    __shared__ bool last;
    red[warp][lane] = part;
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][lane];
        if (valid) a.o.lz.partial[(size_t)blockIdx.x * a.ld + r] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&a.o.lz.counter[blockIdx.y], 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (last && warp == 0) {
        __threadfence();
        double s = 0.0;
        if (valid)
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(&a.o.lz.partial[(size_t)b * a.ld + r]);
        if (valid) a.o.lz.a[(size_t)a.o.k * a.ld + r] = s;
        if (lane == 0) a.o.lz.counter[blockIdx.y] = 0u;
    }
}

template <class T> PrecData<T> &prec(mbd_system *s);
template <> PrecData<double> &prec<double>(mbd_system *s) { return s->f64; }
template <> PrecData<float> &prec<float>(mbd_system *s) { return s->f32; }

Geom geom_of(const mbd_system *s) {
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

}  // namespace

template <class T> mbd_status launch_spread(mbd_system *s, const T *d, T *mesh, int R, int ld) {
    PrecData<T> &P = prec<T>(s);
    SpreadArgs<T> a;
    a.d = d;
    a.mesh = mesh;
    a.R = R;
    a.ld = ld;
    a.g = geom_of(s);
    a.sp = SplineView<T>{s->top_d.as<int>(), P.w.template as<T>(), P.dw.template as<T>(), P.d2w.template as<T>()};
    a.bins = s->bins;
    dim3 grid(s->bins.nb1 * s->bins.nb2 * s->bins.nb3, (R + 31) / 32);
    k_spread<T><<<grid, kWarps * 32, 0, s->stream>>>(a);
    MBD_LAUNCH_CHECK();
    // zero the padded probe columns so that the complex pairing never reads junk
    if (R < ld) {
        MBD_CUDA_TRY(cudaMemset2DAsync(mesh + R, sizeof(T) * ld, 0, sizeof(T) * (ld - R),
                                       (size_t)s->K[0] * s->K[1] * s->K[2], s->stream));
    }
    return MBD_OK;
}

template <class T> mbd_status launch_convolve(mbd_system *s, T *mesh, int ld) {
    using C = typename Cplx<T>::type;
    PrecData<T> &P = prec<T>(s);
    const int V = ld / 2;
    const int K1 = s->K[0], K2 = s->K[1], K3 = s->K[2];
    const int Wmax = sizeof(T) == 4 ? 16 : 8;
    auto run = [&](int dim, int outer, int inner, int sign, bool fused) -> mbd_status {
        FFTArgs<T> a;
        a.data = reinterpret_cast<C *>(mesh);
        a.tw = (dim == 0 ? P.tw1 : (dim == 1 ? P.tw2 : P.tw3)).template as<C>();
        a.G = P.G.template as<T>();
        a.K = s->fft[dim].K;
        a.nst = s->fft[dim].nst;
        for (int k = 0; k < kMaxRadixStages; ++k) a.radix[k] = s->fft[dim].radix[k];
        a.inner = inner;
        a.W = inner < Wmax ? inner : Wmax;
        a.V = V;
        a.sign = sign;
        const size_t smem = 2 * sizeof(C) * (size_t)a.K * a.W;
        dim3 grid((unsigned)((size_t)outer * ((inner + a.W - 1) / a.W)));
        if (fused) {
            if (smem > 48 * 1024)
                MBD_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem));
            k_fft_pass<T, true><<<grid, 256, smem, s->stream>>>(a);
        } else {
            if (smem > 48 * 1024)
                MBD_CUDA_TRY(cudaFuncSetAttribute(k_fft_pass<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)smem));
            k_fft_pass<T, false><<<grid, 256, smem, s->stream>>>(a);
        }
        MBD_LAUNCH_CHECK();
        return MBD_OK;
    };
    MBD_TRY(run(2, K1 * K2, V, -1, false));            // forward along k3
    MBD_TRY(run(1, K1, K3 * V, -1, false));            // forward along k2
    MBD_TRY(run(0, 1, K2 * K3 * V, -1, true));         // forward k1, x G, inverse k1
    MBD_TRY(run(1, K1, K3 * V, +1, false));            // inverse along k2
    MBD_TRY(run(2, K1 * K2, V, +1, false));            // inverse along k3
    return MBD_OK;
}

template <class T>
mbd_status launch_field(mbd_system *s, const T *d, const T *mesh, int R, int ld, const FieldOut<T> &o) {
    PrecData<T> &P = prec<T>(s);
    FieldArgs<T> a;
    a.d = d;
    a.mesh = mesh;
    a.R = R;
    a.ld = ld;
    a.g = geom_of(s);
    a.sp = SplineView<T>{s->top_d.as<int>(), P.w.template as<T>(), P.dw.template as<T>(), P.d2w.template as<T>()};
    a.pr = PairView<T>{s->row_d.as<int>(), s->col_d.as<int>(), s->shift_d.as<int>(), P.pairA.template as<T>()};
    a.order = s->order_d.as<int>();
    a.g_at = s->g_d.as<double>();
    a.w2 = s->w2_d.as<double>();
    a.self_coef = -4.0 * s->ewald_beta * s->ewald_beta * s->ewald_beta / (3.0 * 1.77245385090551602730);
    a.o = o;
    dim3 grid((s->N + kWarps - 1) / kWarps, (R + 31) / 32);
    k_field<T><<<grid, kWarps * 32, 0, s->stream>>>(a);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

int field_blocks(int N) { return (N + kWarps - 1) / kWarps; }

template mbd_status launch_spread<double>(mbd_system *, const double *, double *, int, int);
template mbd_status launch_spread<float>(mbd_system *, const float *, float *, int, int);
template mbd_status launch_convolve<double>(mbd_system *, double *, int);
template mbd_status launch_convolve<float>(mbd_system *, float *, int);
template mbd_status launch_field<double>(mbd_system *, const double *, const double *, int, int,
                                         const FieldOut<double> &);
template mbd_status launch_field<float>(mbd_system *, const float *, const float *, int, int,
                                        const FieldOut<float> &);

}  // namespace mbd
