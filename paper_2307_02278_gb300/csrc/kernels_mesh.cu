// Per-step operator kernels: SPME spreading (Eq. dipolarr), the batched 3D FFT
// convolution with the influence function (Eq. spme), and the fused field
// kernel (SPME gather + real-space pairs + self term, Eqs. spme, fld_ewald,
// fld_ewald1) with the Lanczos epilogue l_k = Omega y_k + Diag(g) E*_k and
// a_k = y_k^T l_k (Eqs. lk3, recurs2).
#include "mbd_internal.cuh"

#include <algorithm>

namespace mbd {

namespace {

constexpr int kWarps = 8;          // warps per block in the field kernel

// Vector loads/stores of VEC consecutive values (VEC in {1, 2, 4}).
template <class T, int VEC> struct VecT;
template <> struct VecT<float, 1> { using type = float; };
template <> struct VecT<float, 2> { using type = float2; };
template <> struct VecT<float, 4> { using type = float4; };
template <> struct VecT<double, 1> { using type = double; };
template <> struct VecT<double, 2> { using type = double2; };

template <class T, int VEC> __device__ __forceinline__ void vload(const T *p, T *v) {
    if constexpr (VEC == 4 && sizeof(T) == 8) {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = b.x;
        v[3] = b.y;
        return;
    } else {
    using V = typename VecT<T, VEC>::type;
    const V x = *reinterpret_cast<const V *>(p);
    if constexpr (VEC == 1) {
        v[0] = x;
    } else if constexpr (VEC == 2) {
        v[0] = x.x;
        v[1] = x.y;
    } else {
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    }
}
template <class T, int VEC> __device__ __forceinline__ void vstore(T *p, const T *v) {
    if constexpr (VEC == 4 && sizeof(T) == 8) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
        return;
    } else {
    using V = typename VecT<T, VEC>::type;
    V x;
    if constexpr (VEC == 1) {
        x = v[0];
    } else if constexpr (VEC == 2) {
        x.x = v[0];
        x.y = v[1];
    } else {
        x.x = v[0];
        x.y = v[1];
        x.z = v[2];
        x.w = v[3];
    }
    *reinterpret_cast<V *>(p) = x;
    }
}

// ---------------------------------------------------------------- spreading
// The dipole array D(k) = sum_j d_j . grad W_j(k) (Eq. dipolarr) is a sparse
// matrix W^T (one row per mesh point, one nonzero per atom whose stencil covers
// the point) times the dense block of dipoles [3N][probes].  W^T is built once
// per geometry in a fixed atom order, so every mesh value is a sum in a fixed
// order: spreading is deterministic and writes each mesh point once.

// Rows of W^T: a thread per mesh point visits the atoms of the bricks whose
// stencils can reach it (binned by their last stencil point) in a fixed order;
// FILL = false counts, FILL = true writes the Cartesian weights
//   dW/dR_alpha = sum_beta C_{beta alpha} dW/du_beta,
//   dW/du = (M'(u1) M(u2) M(u3), M(u1) M'(u2) M(u3), M(u1) M(u2) M'(u3)),
// from FP64 stencil weights.
template <class T, bool FILL>
__global__ void k_spread_rows(Geom g, BinView B, const int *__restrict__ top, const double *__restrict__ w64,
                              const double *__restrict__ dw64, int *__restrict__ cnt_or_row,
                              SpreadRec<T> *__restrict__ rec) {
    const size_t npts = (size_t)g.K1 * g.K2 * g.K3;
    const size_t pt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= npts) return;
    const int g3 = (int)(pt % g.K3), g2 = (int)((pt / g.K3) % g.K2), g1 = (int)(pt / ((size_t)g.K2 * g.K3));
    const int bb1 = g1 / B.bs1, bb2 = g2 / B.bs2, bb3 = g3 / B.bs3;
    const int p = g.p;
    int c = 0;
    const int base = FILL ? cnt_or_row[pt] : 0;
    for (int c1 = 0; c1 < B.nc1; ++c1) {
        const int t1 = (bb1 + c1) % B.nb1;
        for (int c2 = 0; c2 < B.nc2; ++c2) {
            const int t2 = (bb2 + c2) % B.nb2;
            for (int c3 = 0; c3 < B.nc3; ++c3) {
                const int t3 = (bb3 + c3) % B.nb3;
                const int bin = (t1 * B.nb2 + t2) * B.nb3 + t3;
                for (int s = B.start[bin]; s < B.start[bin + 1]; ++s) {
                    const int j = B.atoms[s];
                    int u1 = top[3 * j] - g1;
                    if (u1 < 0) u1 += g.K1;
                    int u2 = top[3 * j + 1] - g2;
                    if (u2 < 0) u2 += g.K2;
                    int u3 = top[3 * j + 2] - g3;
                    if (u3 < 0) u3 += g.K3;
                    if (u1 >= p || u2 >= p || u3 >= p) continue;
                    if (FILL) {
                        const double *w = w64 + (size_t)3 * p * j, *dw = dw64 + (size_t)3 * p * j;
                        const double m1 = w[u1], m2 = w[p + u2], m3 = w[2 * p + u3];
                        const double n1 = dw[u1], n2 = dw[p + u2], n3 = dw[2 * p + u3];
                        const double gu0 = n1 * m2 * m3, gu1 = m1 * n2 * m3, gu2 = m1 * m2 * n3;
                        SpreadRec<T> r;
                        r.w0 = T(g.cmat[0] * gu0 + g.cmat[3] * gu1 + g.cmat[6] * gu2);
                        r.w1 = T(g.cmat[1] * gu0 + g.cmat[4] * gu1 + g.cmat[7] * gu2);
                        r.w2 = T(g.cmat[2] * gu0 + g.cmat[5] * gu1 + g.cmat[8] * gu2);
                        r.atom = j;
                        rec[base + c] = r;
                    }
                    ++c;
                }
            }
        }
    }
    if (!FILL) cnt_or_row[pt] = c;
}

// Exclusive scan of n counts (blocks of 4096), the block sums, and the fix-up.
__global__ void __launch_bounds__(1024) k_scan_block(const int *__restrict__ in, int *__restrict__ out,
                                                     int *__restrict__ bsum, int n) {
    __shared__ int sh[1024];
    const int tid = threadIdx.x;
    const long long base = (long long)blockIdx.x * 4096 + tid * 4;
    int v[4], tsum = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tsum += v[k];
    }
    sh[tid] = tsum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int t = tid >= off ? sh[tid - off] : 0;
        __syncthreads();
        sh[tid] += t;
        __syncthreads();
    }
    int excl = sh[tid] - tsum;
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (tid == 1023) bsum[blockIdx.x] = sh[1023];
}
__global__ void k_scan_sums(int *__restrict__ bsum, int nb, int *__restrict__ total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    long long acc = 0;
    for (int b = 0; b < nb; ++b) {
        const int t = bsum[b];
        bsum[b] = (int)acc;
        acc += t;
    }
    *total = acc > 0x7fffffffLL ? -1 : (int)acc;
}
__global__ void k_scan_add(int *__restrict__ out, const int *__restrict__ bsum, int n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / 4096];
}

// D = W^T d.  A warp takes one mesh point (row) at a time, two rows
// interleaved for memory-level parallelism; lane owns VEC consecutive probes.
// Every lane reads the row's records directly (one broadcast 16-byte load per
// record) and the dipoles with vector loads.  Rows are summed in record order
// (fixed), so the result is deterministic.  Probe columns R..ld-1 (padding of
// an odd probe count) are masked to zero.
template <class T, int VEC>
__global__ void __launch_bounds__(256) k_spread_csr(const T *__restrict__ d, T *__restrict__ mesh, int R, int ld,
                                                    size_t npts, const int *__restrict__ row,
                                                    const SpreadRec<T> *__restrict__ rec) {
    constexpr int U = 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = (blockIdx.y * 32 + lane) * VEC;
    const bool in_ld = r0 < ld;
    const size_t nw = (size_t)gridDim.x * 8;
    T mask[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) mask[v] = (r0 + v < R) ? T(1) : T(0);
    for (size_t pt0 = (size_t)blockIdx.x * 8 + warp; pt0 < npts; pt0 += nw * U) {
        int q[U], qe[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t pt = pt0 + u * nw;
            q[u] = pt < npts ? row[pt] : 0;
            qe[u] = pt < npts ? row[pt + 1] : 0;
        }
        T acc[U][VEC];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[u][v] = T(0);
        bool more = true;
        while (more) {
            more = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q[u] < qe[u]) {
                    const SpreadRec<T> w = rec[q[u]];
                    ++q[u];
                    more = more || q[u] < qe[u];
                    if (in_ld) {
                        T x[VEC], y[VEC], z[VEC];
                        const T *dj = d + (size_t)(3 * w.atom) * ld + r0;
                        vload<T, VEC>(dj, x);
                        vload<T, VEC>(dj + ld, y);
                        vload<T, VEC>(dj + 2 * (size_t)ld, z);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[u][v] += w.w0 * x[v] + w.w1 * y[v] + w.w2 * z[v];
                    }
                }
            }
        }
        if (in_ld) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const size_t pt = pt0 + u * nw;
                if (pt < npts) {
                    T o[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) o[v] = acc[u][v] * mask[v];
                    vstore<T, VEC>(mesh + pt * ld + r0, o);
                }
            }
        }
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
    unsigned long long radices;   // stage s radix = (radices >> 4 s) & 15
    int V;               // complex probe pairs per mesh point (fused pass: G index = e / V)
    int sign;            // -1 forward, +1 inverse (unfused passes)
};

template <class T, class C, int R> __device__ __forceinline__ void dft(C *v, int sign) {
    if constexpr (R == 2) dft2<T>(v);
    else if constexpr (R == 3) dft3<T>(v, sign);
    else if constexpr (R == 4) dft4<T>(v, sign);
    else if constexpr (R == 5) dft5<T>(v, sign);
    else dft8<T>(v, sign);
}

// One radix-R Stockham stage over the K rows of a K x W tile in shared memory
// (R compile-time, so the butterfly stays in registers).
template <class T, class C, int R>
__device__ __forceinline__ void stockham_stage(const C *__restrict__ in, C *__restrict__ out,
                                               const C *__restrict__ tw, int K, int W, int Ns, int sign) {
    const int nb = K / R;
    const int step = K / (Ns * R);
    for (int idx = threadIdx.x; idx < nb * W; idx += blockDim.x) {
        const int j = idx / W, col = idx - j * W;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = in[(j + q * nb) * W + col];
        const int jm = j % Ns;
        if (jm != 0) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C t = tw[q * jm * step];
                if (sign > 0) t.y = -t.y;
                v[q] = cmul(v[q], t);
            }
        }
        dft<T, C, R>(v, sign);
        const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
        for (int q = 0; q < R; ++q) out[(base + q * Ns) * W + col] = v[q];
    }
}

// Mixed-radix Stockham passes over the K rows of a K x W tile held in shared
// memory; returns the buffer that holds the result (natural order).
template <class T, class C>
__device__ C *stockham(C *in, C *out, const FFTArgs<T> &a, const C *tw, int sign) {
    int Ns = 1;
    for (int s = 0; s < a.nst; ++s) {
        const int R = (int)((a.radices >> (4 * s)) & 15ull);
        switch (R) {
            case 2: stockham_stage<T, C, 2>(in, out, tw, a.K, a.W, Ns, sign); break;
            case 3: stockham_stage<T, C, 3>(in, out, tw, a.K, a.W, Ns, sign); break;
            case 4: stockham_stage<T, C, 4>(in, out, tw, a.K, a.W, Ns, sign); break;
            case 5: stockham_stage<T, C, 5>(in, out, tw, a.K, a.W, Ns, sign); break;
            default: stockham_stage<T, C, 8>(in, out, tw, a.K, a.W, Ns, sign); break;
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
    C *tw = b1 + a.K * a.W;
    for (int i = threadIdx.x; i < a.K; i += blockDim.x) tw[i] = a.tw[i];
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
        res = stockham<T, C>(b0, b1, a, tw, -1);
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
        res = stockham<T, C>(res, other, a, tw, +1);
    } else {
        res = stockham<T, C>(b0, b1, a, tw, a.sign);
    }
    for (int idx = threadIdx.x; idx < a.K * a.W; idx += blockDim.x) {
        const int row = idx / a.W, col = idx - row * a.W;
        if (col < wc) base[(size_t)row * a.inner + col] = res[idx];
    }
}

// Compile-time specialisation of the pass for common mesh sizes: K, the
// radix list, the tile width W and every stride are constants, so the index
// arithmetic folds away and each stage is one unrolled butterfly per thread.
template <class T, class C, int R, int K, int W, int NS, bool IN_G, bool OUT_G, bool MULG>
__device__ __forceinline__ void ct_stage(const C *__restrict__ in_s, const C *__restrict__ in_g, C *__restrict__ out_s,
                                         C *__restrict__ out_g, size_t gs, int wc, const C *__restrict__ tw, int sign,
                                         const T *__restrict__ G, size_t gstride, int c0, int V) {
    constexpr int nb = K / R;
    constexpr int step = K / (NS * R);
    constexpr int total = nb * W;
#pragma unroll
    for (int it = 0; it < (total + 255) / 256; ++it) {
        const int idx = it * 256 + (int)threadIdx.x;
        if (total % 256 != 0 && idx >= total) break;
        const int j = idx / W, col = idx % W;
        C v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (IN_G)
                v[q] = col < wc ? in_g[(size_t)(j + q * nb) * gs + col] : C{T(0), T(0)};
            else
                v[q] = in_s[(j + q * nb) * W + col];
        }
        const int jm = j % NS;
        if (NS > 1 && jm != 0) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C t = tw[q * jm * step];
                if (sign > 0) t.y = -t.y;
                v[q] = cmul(v[q], t);
            }
        }
        dft<T, C, R>(v, sign);
        const int base = (j / NS) * NS * R + jm;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = base + q * NS;
            if (MULG && col < wc) {
                const T gv = G[(size_t)row * gstride + (c0 + col) / V];
                v[q].x *= gv;
                v[q].y *= gv;
            }
            if (OUT_G) {
                if (col < wc) out_g[(size_t)row * gs + col] = v[q];
            } else {
                out_s[row * W + col] = v[q];
            }
        }
    }
}

// A run of Stockham stages: the first reads the global tile (IN_G) or shared
// buffer sin, intermediate results ping-pong between sin and sout, the last
// writes the global tile (OUT_G) or shared memory, multiplying by G (MULG).
// Returns the shared buffer holding the result when it stays in shared memory.
template <class T, class C, int K, int W, int NS, bool IN_G, bool OUT_G, bool MULG, int R, int... RS>
__device__ __forceinline__ C *ct_pipe(const C *gin, C *gout, size_t gs, int wc, C *sin, C *sout, const C *tw, int sign,
                                      const T *G, size_t gstride, int c0, int V) {
    constexpr bool last = sizeof...(RS) == 0;
    ct_stage<T, C, R, K, W, NS, IN_G, last && OUT_G, last && MULG>(sin, gin, sout, gout, gs, wc, tw, sign, G, gstride,
                                                                   c0, V);
    if constexpr (last) {
        return sout;
    } else {
        __syncthreads();
        return ct_pipe<T, C, K, W, NS * R, false, OUT_G, MULG, RS...>(gin, gout, gs, wc, sout, sin, tw, sign, G, gstride,
                                                                       c0, V);
    }
}

// One pass with compile-time K, W and radices (at least two stages).  The
// first stage loads the global tile straight into registers and the last one
// stores straight from registers, so shared memory carries only the exchanges
// between stages; the fused pass (forward, x G, inverse) multiplies by G in the
// last forward stage.
template <class T, bool FUSED, int K, int W, int... RS>
__global__ void __launch_bounds__(256) k_fft_ct(FFTArgs<T> a) {
    using C = typename Cplx<T>::type;
    static_assert(sizeof...(RS) >= 2, "single-stage sizes would read and write the same global tile");
    extern __shared__ __align__(16) unsigned char smem_ct[];
    C *buf0 = reinterpret_cast<C *>(smem_ct), *buf1 = buf0 + K * W;
    C *tw = buf1 + K * W;
    for (int i = threadIdx.x; i < K; i += 256) tw[i] = a.tw[i];
    __syncthreads();
    const int ncb = (a.inner + W - 1) / W;
    const size_t outer = blockIdx.x / ncb;
    const int c0 = (int)(blockIdx.x % ncb) * W;
    const int wc = min(W, a.inner - c0);
    C *base = a.data + outer * (size_t)K * a.inner + c0;
    const size_t gstride = (size_t)(a.inner / a.V);
    if (FUSED) {
        C *res = ct_pipe<T, C, K, W, 1, true, false, true, RS...>(base, base, a.inner, wc, buf0, buf1, tw, -1, a.G,
                                                                   gstride, c0, a.V);
        __syncthreads();
        C *other = (res == buf0) ? buf1 : buf0;
        ct_pipe<T, C, K, W, 1, false, true, false, RS...>(base, base, a.inner, wc, res, other, tw, +1, a.G, gstride, c0,
                                                           a.V);
    } else {
        ct_pipe<T, C, K, W, 1, true, true, false, RS...>(base, base, a.inner, wc, buf0, buf1, tw, a.sign, a.G, gstride,
                                                          c0, a.V);
    }
}

template <class T, bool FUSED, int K, int W, int... RS>
bool launch_ct(const FFTArgs<T> &a, unsigned grid, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const size_t smem = sizeof(C) * (2 * (size_t)K * W + K);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_fft_ct<T, FUSED, K, W, RS...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    k_fft_ct<T, FUSED, K, W, RS...><<<grid, 256, smem, st>>>(a);
    return true;
}

// Spreading fused with the forward FFT along k3: a block owns one (k1, k2)
// pencil of K3 mesh points and W complex probe-pair columns.  Warp w spreads
// rows k3 = w, w + 8, ... straight into the shared-memory tile (same records
// and order as k_spread_csr), then the block transforms the tile along k3 and
// writes it once.  Probe columns >= R are masked to zero.
template <class T, int K, int W, int... RS>
__global__ void __launch_bounds__(256) k_spread_fft3(const T *__restrict__ d, typename Cplx<T>::type *__restrict__ mesh,
                                                     int R, int ld, int K2, const int *__restrict__ row,
                                                     const SpreadRec<T> *__restrict__ rec,
                                                     const typename Cplx<T>::type *__restrict__ twg) {
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_sf[];
    C *buf0 = reinterpret_cast<C *>(smem_sf);
    C *buf1 = buf0 + K * W;
    C *tw = buf1 + K * W;
    for (int i = threadIdx.x; i < K; i += 256) tw[i] = twg[i];
    const int V = ld / 2;
    const int ncb = (V + W - 1) / W;
    const size_t pencil = blockIdx.x / ncb;              // k1 * K2 + k2
    const int c0 = (int)(blockIdx.x % ncb) * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = c0 + lane;                           // complex column = probes 2 col, 2 col + 1
    const bool on = lane < W && col < V;
    const T m0 = (2 * col < R) ? T(1) : T(0), m1 = (2 * col + 1 < R) ? T(1) : T(0);
    // two rows (k3 and k3 + 8) per warp iteration: two independent load chains
    for (int k3 = warp; k3 < K; k3 += 16) {
        const int kb = k3 + 8;
        const size_t pa = pencil * K + k3, pb = pencil * K + kb;
        int qa = row[pa];
        const int qa1 = row[pa + 1];
        int qb = 0, qb1 = 0;
        if (kb < K) {
            qb = row[pb];
            qb1 = row[pb + 1];
        }
        T ax = T(0), ay = T(0), bx = T(0), by = T(0);
        while (qa < qa1 || qb < qb1) {
            if (qa < qa1) {
                const SpreadRec<T> w = rec[qa++];
                if (on) {
                    T x[2], y[2], z[2];
                    const T *dj = d + (size_t)(3 * w.atom) * ld + 2 * col;
                    vload<T, 2>(dj, x);
                    vload<T, 2>(dj + ld, y);
                    vload<T, 2>(dj + 2 * (size_t)ld, z);
                    ax += w.w0 * x[0] + w.w1 * y[0] + w.w2 * z[0];
                    ay += w.w0 * x[1] + w.w1 * y[1] + w.w2 * z[1];
                }
            }
            if (qb < qb1) {
                const SpreadRec<T> w = rec[qb++];
                if (on) {
                    T x[2], y[2], z[2];
                    const T *dj = d + (size_t)(3 * w.atom) * ld + 2 * col;
                    vload<T, 2>(dj, x);
                    vload<T, 2>(dj + ld, y);
                    vload<T, 2>(dj + 2 * (size_t)ld, z);
                    bx += w.w0 * x[0] + w.w1 * y[0] + w.w2 * z[0];
                    by += w.w0 * x[1] + w.w1 * y[1] + w.w2 * z[1];
                }
            }
        }
        if (lane < W) {
            buf0[k3 * W + lane] = on ? C{ax * m0, ay * m1} : C{T(0), T(0)};
            if (kb < K) buf0[kb * W + lane] = on ? C{bx * m0, by * m1} : C{T(0), T(0)};
        }
    }
    __syncthreads();
    const int wc = min(W, V - c0);
    C *base = mesh + pencil * (size_t)K * V + c0;
    ct_pipe<T, C, K, W, 1, false, true, false, RS...>(base, base, (size_t)V, wc, buf0, buf1, tw, -1,
                                                       (const T *)nullptr, 0, c0, V);
}

template <class T, int K, int W, int... RS>
bool launch_sf3(const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row, const SpreadRec<T> *rec,
                const typename Cplx<T>::type *tw, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    const size_t smem = sizeof(C) * (2 * (size_t)K * W + K);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_spread_fft3<T, K, W, RS...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    const int V = ld / 2;
    const unsigned grid = (unsigned)((size_t)K1 * K2 * ((V + W - 1) / W));
    k_spread_fft3<T, K, W, RS...><<<grid, 256, smem, st>>>(d, reinterpret_cast<C *>(mesh), R, ld, K2, row, rec, tw);
    return true;
}

// Launch the specialised pass when K has one; returns false otherwise.
template <class T, bool FUSED>
bool launch_fft_ct(const FFTArgs<T> &a, unsigned grid, cudaStream_t st) {
    constexpr int W = sizeof(T) == 4 ? 32 : 16;
    if (a.W != W) return false;
    switch (a.K) {
        case 32: return launch_ct<T, FUSED, 32, W, 8, 4>(a, grid, st);
        case 64: return launch_ct<T, FUSED, 64, W, 8, 8>(a, grid, st);
        case 96: return launch_ct<T, FUSED, 96, W, 8, 4, 3>(a, grid, st);
        case 128: return launch_ct<T, FUSED, 128, W, 8, 8, 2>(a, grid, st);
        case 192: return launch_ct<T, FUSED, 192, W, 8, 8, 3>(a, grid, st);
        default: return false;
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

// Field kernel: one block works on `apb` atoms in turn; for each atom its 8
// warps split the work (warp w takes stencil planes t1 = w, w + 8, ... and
// neighbours nb0 + w, nb0 + w + 8, ...; warp 0 adds the self term), lanes own
// VEC consecutive probes.  The 8 partial fields are summed in a fixed order in
// shared memory and the epilogue selected by o.mode runs with one thread per
// probe: E* = E^rec + E^dir + E^self (Eqs. ewalddip, spme, fld_ewald,
// fld_ewald1), l_k = Omega y_k + Diag(g) E*_k and a_k = y_k^T l_k (Eqs. lk3,
// recurs2).  PC = spline order (0: runtime).
template <class T, int VEC, int PC>
__global__ void __launch_bounds__(kWarps * 32, (VEC <= 2 && sizeof(T) == 4 && PC > 0) ? 3 : 2)
    k_field(FieldArgs<T> a, int apb) {
    constexpr int NLOC = 32 * VEC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rbase = blockIdx.y * NLOC;
    const int r0 = rbase + lane * VEC;
    const bool inld = r0 < a.ld;
    const int p = PC > 0 ? PC : a.g.p;
    __shared__ T red[kWarps][3][NLOC];
    __shared__ double bsum[NLOC];
    __shared__ double pcarry[3 * NLOC > kWarps * 32 ? 3 * NLOC - kWarps * 32 : 1];
    __shared__ double pall[3 * NLOC];
    for (int k = threadIdx.x; k < (3 * NLOC > kWarps * 32 ? 3 * NLOC - kWarps * 32 : 1); k += blockDim.x)
        pcarry[k] = 0.0;
    double part = 0.0;                          // y.l of the (component, probe) this thread owns
    for (int ai = 0; ai < apb; ++ai) {
        const int idx = blockIdx.x * apb + ai;
        if (idx >= a.g.N) break;
        const int i = a.order[idx];
        T E0[VEC], E1[VEC], E2[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) E0[v] = E1[v] = E2[v] = T(0);
        if (inld) {
            if (a.o.terms & MBD_TERM_RECIP) {
                T f0[VEC], f1[VEC], f2[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) f0[v] = f1[v] = f2[v] = T(0);
                const int top1 = a.sp.top[3 * i], top2 = a.sp.top[3 * i + 1], top3 = a.sp.top[3 * i + 2];
                const T *w = a.sp.w + (size_t)3 * p * i;
                const T *dw = a.sp.dw + (size_t)3 * p * i;
                for (int t1 = warp; t1 < p; t1 += kWarps) {
                    int k1 = top1 - t1;
                    if (k1 < 0) k1 += a.g.K1;
                    const T wa = w[t1], da = dw[t1];
#pragma unroll
                    for (int t2 = 0; t2 < (PC > 0 ? PC : kMaxOrder); ++t2) {
                        if (t2 >= p) break;
                        int k2 = top2 - t2;
                        if (k2 < 0) k2 += a.g.K2;
                        const T wb = w[p + t2], db = dw[p + t2];
                        const T ab = wa * wb, Ab = da * wb, aB = wa * db;
                        const T *rowp = a.mesh + ((size_t)k1 * a.g.K2 + k2) * a.g.K3 * a.ld + r0;
#pragma unroll
                        for (int t3 = 0; t3 < (PC > 0 ? PC : kMaxOrder); ++t3) {
                            if (t3 >= p) break;
                            int k3 = top3 - t3;
                            if (k3 < 0) k3 += a.g.K3;
                            T phi[VEC];
                            vload<T, VEC>(rowp + (size_t)k3 * a.ld, phi);
                            const T wc = w[2 * p + t3], dc = dw[2 * p + t3];
                            const T c0 = Ab * wc, c1 = aB * wc, c2 = ab * dc;
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                f0[v] += c0 * phi[v];
                                f1[v] += c1 * phi[v];
                                f2[v] += c2 * phi[v];
                            }
                        }
                    }
                }
                // E^rec_alpha = sum_beta C_{beta alpha} f_beta
                const T m00 = T(a.g.cmat[0]), m01 = T(a.g.cmat[1]), m02 = T(a.g.cmat[2]);
                const T m10 = T(a.g.cmat[3]), m11 = T(a.g.cmat[4]), m12 = T(a.g.cmat[5]);
                const T m20 = T(a.g.cmat[6]), m21 = T(a.g.cmat[7]), m22 = T(a.g.cmat[8]);
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    E0[v] += m00 * f0[v] + m10 * f1[v] + m20 * f2[v];
                    E1[v] += m01 * f0[v] + m11 * f1[v] + m21 * f2[v];
                    E2[v] += m02 * f0[v] + m12 * f1[v] + m22 * f2[v];
                }
            }
            if (a.o.terms & MBD_TERM_REAL) {
                const int nb1 = a.pr.row[i + 1];
                constexpr int B4 = 4;
                for (int nb = a.pr.row[i] + warp; nb < nb1; nb += B4 * kWarps) {
                    int jj[B4];
#pragma unroll
                    for (int u = 0; u < B4; ++u) jj[u] = (nb + u * kWarps < nb1) ? a.pr.col[nb + u * kWarps] : -1;
                    T xs[B4][VEC], ys[B4][VEC], zs[B4][VEC];
#pragma unroll
                    for (int u = 0; u < B4; ++u) {
                        if (jj[u] >= 0) {
                            const T *dj = a.d + (size_t)(3 * jj[u]) * a.ld + r0;
                            vload<T, VEC>(dj, xs[u]);
                            vload<T, VEC>(dj + a.ld, ys[u]);
                            vload<T, VEC>(dj + 2 * (size_t)a.ld, zs[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < B4; ++u) {
                        if (jj[u] >= 0) {
                            const T *A = a.pr.A + 6 * (size_t)(nb + u * kWarps);
                            const T A0 = A[0], A1 = A[1], A2 = A[2], A3 = A[3], A4 = A[4], A5 = A[5];
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                E0[v] += A0 * xs[u][v] + A1 * ys[u][v] + A2 * zs[u][v];
                                E1[v] += A1 * xs[u][v] + A3 * ys[u][v] + A4 * zs[u][v];
                                E2[v] += A2 * xs[u][v] + A4 * ys[u][v] + A5 * zs[u][v];
                            }
                        }
                    }
                }
            }
            if ((a.o.terms & MBD_TERM_SELF) && warp == 0) {
                const T c = T(a.self_coef);
                T x[VEC], y[VEC], z[VEC];
                const T *di = a.d + (size_t)(3 * i) * a.ld + r0;
                vload<T, VEC>(di, x);
                vload<T, VEC>(di + a.ld, y);
                vload<T, VEC>(di + 2 * (size_t)a.ld, z);
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    E0[v] += c * x[v];
                    E1[v] += c * y[v];
                    E2[v] += c * z[v];
                }
            }
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            red[warp][0][lane * VEC + v] = E0[v];
            red[warp][1][lane * VEC + v] = E1[v];
            red[warp][2][lane * VEC + v] = E2[v];
        }
        __syncthreads();
        // epilogue: one thread per (component, probe) so that the FP64 work
        // spreads over 6 warps
        for (int cp = threadIdx.x; cp < 3 * NLOC; cp += blockDim.x) {
            const int c = cp / NLOC, t = cp - c * NLOC;
            const int r = rbase + t;
            if (r < a.ld) {
                T sum = T(0);
#pragma unroll
                for (int w = 0; w < kWarps; ++w) sum += red[w][c][t];
                const double E = double(sum);
                const size_t o = (size_t)(3 * i + c) * a.ld + r;
                if (a.o.mode == kFieldOut) {
                    a.o.out[o] = E;
                } else if (a.o.mode == kFieldApply) {
                    a.o.out[o] = a.w2[i] * a.o.xin[o] + a.g_at[i] * E;
                } else {
                    const double invb = a.o.lz.invb[r];
                    double *Yk = a.o.lz.Y + (size_t)a.o.k * (size_t)(3 * a.g.N) * a.ld;
                    const double y = Yk[o] * invb;
                    const double l = a.w2[i] * y + a.g_at[i] * E * invb;
                    Yk[o] = y;
                    a.o.lz.L[o] = l;
                    if (cp < (int)blockDim.x) part += y * l;
                    else pcarry[cp - blockDim.x] += y * l;   // thread cp - blockDim.x owns this slot
                }
            }
        }
        __syncthreads();
    }
    if (a.o.mode != kFieldLanczos) return;
    // a_k = y_k^T l_k: per probe, the three components in order, then a
    // deterministic reduction over blocks
    for (int cp = threadIdx.x; cp < 3 * NLOC; cp += blockDim.x)
        pall[cp] = (cp < (int)blockDim.x) ? part : pcarry[cp - blockDim.x];
    __syncthreads();
    for (int t = threadIdx.x; t < NLOC; t += blockDim.x) bsum[t] = pall[t] + pall[NLOC + t] + pall[2 * NLOC + t];
    __syncthreads();
    __shared__ double tot[NLOC];
    if (grid_reduce(bsum, NLOC, rbase, a.R, a.ld, a.o.lz, tot)) {
        for (int k = threadIdx.x; k < NLOC; k += blockDim.x)
            if (rbase + k < a.R) a.o.lz.a[(size_t)a.o.k * a.ld + rbase + k] = tot[k];
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

template <class T> mbd_status build_spread_matrix(mbd_system *s) {
    PrecData<T> &P = prec<T>(s);
    const Geom g = geom_of(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    if (npts >= 0x7fffffffULL) return MBD_ERR_UNSUPPORTED;
    MBD_TRY(P.srow.ensure(sizeof(int) * (npts + 1)));
    DevBuf cnt, bsum, total;
    const int n = (int)npts;
    const int nb = (n + 4095) / 4096;
    MBD_TRY(cnt.ensure(sizeof(int) * npts));
    MBD_TRY(bsum.ensure(sizeof(int) * nb));
    MBD_TRY(total.ensure(sizeof(int)));
    const int threads = 256;
    const unsigned blocks = (unsigned)((npts + threads - 1) / threads);
    k_spread_rows<T, false><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                              s->dw64_d.as<double>(), cnt.as<int>(), nullptr);
    MBD_LAUNCH_CHECK();
    k_scan_block<<<nb, 1024, 0, s->stream>>>(cnt.as<int>(), P.srow.template as<int>(), bsum.as<int>(), n);
    MBD_LAUNCH_CHECK();
    k_scan_sums<<<1, 32, 0, s->stream>>>(bsum.as<int>(), nb, P.srow.template as<int>() + n);
    MBD_LAUNCH_CHECK();
    k_scan_add<<<(n + 255) / 256, 256, 0, s->stream>>>(P.srow.template as<int>(), bsum.as<int>(), n);
    MBD_LAUNCH_CHECK();
    int nnz = 0;
    MBD_CUDA_TRY(cudaMemcpyAsync(&nnz, P.srow.template as<int>() + n, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (nnz < 0) return MBD_ERR_UNSUPPORTED;
    MBD_TRY(P.srec.ensure(sizeof(SpreadRec<T>) * (size_t)(nnz > 0 ? nnz : 1)));
    k_spread_rows<T, true><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                             s->dw64_d.as<double>(), P.srow.template as<int>(),
                                                             P.srec.template as<SpreadRec<T>>());
    MBD_LAUNCH_CHECK();
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));   // cnt, bsum, total are freed on return
    return MBD_OK;
}

template <class T> mbd_status launch_spread(mbd_system *s, const T *d, T *mesh, int R, int ld) {
    PrecData<T> &P = prec<T>(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    const int vec = (sizeof(T) == 4 && ld % 4 == 0 && ld >= 128) ? 4 : ((ld % 2 == 0 && ld >= 64) ? 2 : 1);
    const unsigned gx = (unsigned)std::min<size_t>((npts + 15) / 16, 152 * 16);
    dim3 grid(gx, (ld + 32 * vec - 1) / (32 * vec));
    const int *rowp = P.srow.template as<int>();
    const SpreadRec<T> *recp = P.srec.template as<SpreadRec<T>>();
    if (vec == 4) {
        if constexpr (sizeof(T) == 4) k_spread_csr<T, 4><<<grid, 256, 0, s->stream>>>(d, mesh, R, ld, npts, rowp, recp);
    } else if (vec == 2) {
        k_spread_csr<T, 2><<<grid, 256, 0, s->stream>>>(d, mesh, R, ld, npts, rowp, recp);
    } else {
        k_spread_csr<T, 1><<<grid, 256, 0, s->stream>>>(d, mesh, R, ld, npts, rowp, recp);
    }
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

// Spreading fused with the first forward FFT pass when the k3 size has a
// specialised pass and the probe-pair columns fill whole tiles; returns
// MBD_ERR_UNSUPPORTED (nothing launched) otherwise.
bool spread_fft3_supported(int K3, int ld, int real_bytes) {
    const int W = real_bytes == 4 ? 32 : 16;
    const bool k_ok = K3 == 32 || K3 == 64 || K3 == 96 || K3 == 128 || K3 == 192;
    return k_ok && (ld / 2) % W == 0;
}

template <class T> mbd_status launch_spread_fft3(mbd_system *s, const T *d, T *mesh, int R, int ld) {
    PrecData<T> &P = prec<T>(s);
    constexpr int W = sizeof(T) == 4 ? 32 : 16;
    const int V = ld / 2;
    if (V % W != 0) return MBD_ERR_UNSUPPORTED;
    using C = typename Cplx<T>::type;
    const int *row = P.srow.template as<int>();
    const SpreadRec<T> *rec = P.srec.template as<SpreadRec<T>>();
    const C *tw = P.tw3.template as<C>();
    bool ok = false;
    switch (s->K[2]) {
        case 32: ok = launch_sf3<T, 32, W, 8, 4>(d, mesh, R, ld, s->K[0], s->K[1], row, rec, tw, s->stream); break;
        case 64: ok = launch_sf3<T, 64, W, 8, 8>(d, mesh, R, ld, s->K[0], s->K[1], row, rec, tw, s->stream); break;
        case 96: ok = launch_sf3<T, 96, W, 8, 4, 3>(d, mesh, R, ld, s->K[0], s->K[1], row, rec, tw, s->stream); break;
        case 128: ok = launch_sf3<T, 128, W, 8, 8, 2>(d, mesh, R, ld, s->K[0], s->K[1], row, rec, tw, s->stream); break;
        case 192: ok = launch_sf3<T, 192, W, 8, 8, 3>(d, mesh, R, ld, s->K[0], s->K[1], row, rec, tw, s->stream); break;
        default: ok = false;
    }
    if (!ok) return MBD_ERR_UNSUPPORTED;
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T> mbd_status launch_convolve(mbd_system *s, T *mesh, int ld, bool skip_first) {
    using C = typename Cplx<T>::type;
    PrecData<T> &P = prec<T>(s);
    const int V = ld / 2;
    const int K1 = s->K[0], K2 = s->K[1], K3 = s->K[2];
    const int Wmax = sizeof(T) == 4 ? 32 : 16;
    auto run = [&](int dim, int outer, int inner, int sign, bool fused) -> mbd_status {
        FFTArgs<T> a;
        a.data = reinterpret_cast<C *>(mesh);
        a.tw = (dim == 0 ? P.tw1 : (dim == 1 ? P.tw2 : P.tw3)).template as<C>();
        a.G = P.G.template as<T>();
        a.K = s->fft[dim].K;
        a.nst = s->fft[dim].nst;
        a.radices = 0ull;
        for (int k = 0; k < a.nst; ++k) a.radices |= (unsigned long long)s->fft[dim].radix[k] << (4 * k);
        a.inner = inner;
        a.W = inner < Wmax ? inner : Wmax;
        a.V = V;
        a.sign = sign;
        const size_t smem = sizeof(C) * (2 * (size_t)a.K * a.W + a.K);
        dim3 grid((unsigned)((size_t)outer * ((inner + a.W - 1) / a.W)));
        if (fused ? launch_fft_ct<T, true>(a, grid.x, s->stream) : launch_fft_ct<T, false>(a, grid.x, s->stream)) {
            MBD_LAUNCH_CHECK();
            return MBD_OK;
        }
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
    if (!skip_first) MBD_TRY(run(2, K1 * K2, V, -1, false));   // forward along k3
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
    const int vec = (sizeof(T) == 4 && ld % 4 == 0 && ld >= 128) ? 4 : ((ld % 2 == 0 && ld >= 64) ? 2 : 1);
    const int apb = field_apb(s->N);
    dim3 grid(field_blocks(s->N), (ld + 32 * vec - 1) / (32 * vec));
#define MBD_FIELD_LAUNCH(V, P) k_field<T, V, P><<<grid, kWarps * 32, 0, s->stream>>>(a, apb)
    if (vec == 4) {
        if constexpr (sizeof(T) == 4) {
            if (s->p == 6) MBD_FIELD_LAUNCH(4, 6);
            else MBD_FIELD_LAUNCH(4, 0);
        }
    } else if (vec == 2) {
        if (s->p == 6) MBD_FIELD_LAUNCH(2, 6);
        else MBD_FIELD_LAUNCH(2, 0);
    } else {
        if (s->p == 6) MBD_FIELD_LAUNCH(1, 6);
        else MBD_FIELD_LAUNCH(1, 0);
    }
#undef MBD_FIELD_LAUNCH
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

// Atoms per block of the field kernel: about four blocks per SM.
int field_apb(int N) { return std::max(1, std::min(64, (N + 152 * 4 - 1) / (152 * 4))); }
int field_blocks(int N) { return (N + field_apb(N) - 1) / field_apb(N); }

template mbd_status build_spread_matrix<double>(mbd_system *);
template mbd_status build_spread_matrix<float>(mbd_system *);
template mbd_status launch_spread<double>(mbd_system *, const double *, double *, int, int);
template mbd_status launch_spread<float>(mbd_system *, const float *, float *, int, int);
template mbd_status launch_convolve<double>(mbd_system *, double *, int, bool);
template mbd_status launch_convolve<float>(mbd_system *, float *, int, bool);
template mbd_status launch_spread_fft3<double>(mbd_system *, const double *, double *, int, int);
template mbd_status launch_spread_fft3<float>(mbd_system *, const float *, float *, int, int);
template mbd_status launch_field<double>(mbd_system *, const double *, const double *, int, int,
                                         const FieldOut<double> &);
template mbd_status launch_field<float>(mbd_system *, const float *, const float *, int, int,
                                        const FieldOut<float> &);

}  // namespace mbd
