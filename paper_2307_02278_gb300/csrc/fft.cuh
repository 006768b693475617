// Mesh-stage device code shared by the operator kernels (kernels_mesh.cu) and
// the compile-time FFT passes (fft_sizes_*.cu): vector loads, complex
// arithmetic, the in-register DFTs, the Stockham passes with compile-time
// mesh size, and the spreading fused with the first forward pass.
#pragma once

#include <algorithm>

#include "mbd_internal.cuh"

namespace mbd {

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
    int early;           // compile-time passes: programmatic dependent launch (1) or plain (0)
    int sms;             // multiprocessors (persistent compile-time passes; 0: not persistent)
};

// Compile-time passes for the smooth sizes listed below (fft_sizes_*.cu).
// Return 1 when launched, 0 when the launch could not be configured, -1 when
// there is no compile-time pass for the size or tile width asked for.
//   a.W: the tile width; float passes exist for W = 32 and 16, double
//   passes for W = 16.
template <class T> int launch_fft_ct_sized(const FFTArgs<T> &a, bool fused, unsigned grid, cudaStream_t st);
//   W: the tile width of the fused spreading (float 32 or 16, double 16).
template <class T>
int launch_sf3_sized(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row,
                     const SpreadRec<T> *rec, const typename Cplx<T>::type *tw, cudaStream_t st);
bool fft_ct_size(int K);
//   The same fused pass with spreading by pencil records (spline order 6):
//   W = 32 or 16 for float, 16 for double.
template <class T>
int launch_spp_sized(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow,
                     const PencilRec<T> *prec, const T *k3w, const typename Cplx<T>::type *tw, cudaStream_t st);

// Sizes with a compile-time pass and their radices (first stage first), in
// groups of one translation unit each.
#define MBD_FFT_GROUP0(X) X(16, 4, 4) X(18, 3, 3, 2) X(20, 5, 4) X(24, 8, 3) X(25, 5, 5) X(27, 3, 3, 3) X(30, 5, 3, 2)
#define MBD_FFT_GROUP1(X) X(32, 8, 4) X(36, 4, 3, 3) X(40, 8, 5) X(45, 5, 3, 3) X(48, 4, 4, 3) X(50, 5, 5, 2) \
    X(54, 3, 3, 3, 2)
#define MBD_FFT_GROUP2(X) X(60, 5, 4, 3) X(64, 8, 8) X(72, 8, 3, 3) X(75, 5, 5, 3) X(80, 5, 4, 4) \
    X(81, 3, 3, 3, 3) X(90, 5, 3, 3, 2)
#define MBD_FFT_GROUP3(X) X(96, 8, 4, 3) X(100, 5, 5, 4) X(108, 4, 3, 3, 3) X(120, 8, 5, 3) X(125, 5, 5, 5) \
    X(128, 8, 8, 2) X(135, 5, 3, 3, 3)
#define MBD_FFT_GROUP4(X) X(144, 4, 4, 3, 3) X(150, 5, 5, 3, 2) X(160, 8, 5, 4) X(162, 3, 3, 3, 3, 2) \
    X(180, 5, 4, 3, 3) X(192, 8, 8, 3) X(200, 8, 5, 5)
#define MBD_FFT_GROUP5(X) X(216, 8, 3, 3, 3) X(225, 5, 5, 3, 3) X(240, 5, 4, 4, 3) X(243, 3, 3, 3, 3, 3) \
    X(250, 5, 5, 5, 2) X(256, 8, 8, 4)
#define MBD_FFT_NUM_GROUPS 6

template <class T> int launch_fft_ct_group0(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
template <class T> int launch_fft_ct_group1(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
template <class T> int launch_fft_ct_group2(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
template <class T> int launch_fft_ct_group3(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
template <class T> int launch_fft_ct_group4(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
template <class T> int launch_fft_ct_group5(const FFTArgs<T> &, bool, unsigned, cudaStream_t);
#define MBD_SF3_DECL(g)                                                                                          \
    template <class T>                                                                                           \
    int launch_sf3_group##g(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row, \
                            const SpreadRec<T> *rec, const typename Cplx<T>::type *tw, cudaStream_t st);
MBD_SF3_DECL(0)
MBD_SF3_DECL(1)
MBD_SF3_DECL(2)
MBD_SF3_DECL(3)
MBD_SF3_DECL(4)
MBD_SF3_DECL(5)
#undef MBD_SF3_DECL
#define MBD_SPP_DECL(g)                                                                                          \
    template <class T>                                                                                           \
    int launch_spp_group##g(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow, \
                            const PencilRec<T> *prec, const T *k3w, const typename Cplx<T>::type *tw,            \
                            cudaStream_t st);
MBD_SPP_DECL(0)
MBD_SPP_DECL(1)
MBD_SPP_DECL(2)
MBD_SPP_DECL(3)
MBD_SPP_DECL(4)
MBD_SPP_DECL(5)
#undef MBD_SPP_DECL

namespace {

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



template <class T, class C, int R> __device__ __forceinline__ void dft(C *v, int sign) {
    if constexpr (R == 2) dft2<T>(v);
    else if constexpr (R == 3) dft3<T>(v, sign);
    else if constexpr (R == 4) dft4<T>(v, sign);
    else if constexpr (R == 5) dft5<T>(v, sign);
    else dft8<T>(v, sign);
}

// ---------------------------------------------------------------- compile-time passes
// Threads of a compile-time pass: enough for the stage with the most
// butterflies (K / smallest radix rows x W columns), at most 256.
template <int R> constexpr int ct_rmin() { return R; }
template <int R, int S, int... RS> constexpr int ct_rmin() {
    return R < ct_rmin<S, RS...>() ? R : ct_rmin<S, RS...>();
}
template <int K, int W, int... RS> constexpr int ct_threads() {
    return (K / ct_rmin<RS...>()) * W >= 256 ? 256 : (((K / ct_rmin<RS...>()) * W + 31) / 32) * 32;
}

// One radix-R Stockham stage over the K rows of a K x W tile with K, W, the
// stage's stride NS and the block size NT compile-time, so the index
// arithmetic folds away and each butterfly stays in registers.  The stage reads
// the global tile (IN_G, columns >= wc read as zero) or shared memory, and
// writes the global tile (OUT_G, columns < wc only) or shared memory,
// multiplying by G on the way out (MULG; G index row * gstride + (c0 + col) / V).
// A thread takes CV adjacent columns of a row (CV = 2: float tiles, one
// 16-byte access for both and one twiddle for both; the caller guarantees
// whole column pairs, 16-byte alignment and an even V).
template <class T, class C, int R, int K, int W, int NT, int CV, int NS, bool IN_G, bool OUT_G, bool MULG>
__device__ __forceinline__ void ct_stage(const C *__restrict__ in_s, const C *__restrict__ in_g, C *__restrict__ out_s,
                                         C *__restrict__ out_g, size_t gs, int wc, const C *__restrict__ tw, int sign,
                                         const T *__restrict__ G, size_t gstride, int c0, int V) {
    static_assert(CV == 1 || (CV == 2 && sizeof(T) == 4 && W % 2 == 0), "column pairs are float tiles");
    constexpr int nb = K / R;
    constexpr int step = K / (NS * R);
    constexpr int WG = W / CV;
    constexpr int total = nb * WG;
#pragma unroll
    for (int it = 0; it < (total + NT - 1) / NT; ++it) {
        const int idx = it * NT + (int)threadIdx.x;
        if (total % NT != 0 && idx >= total) break;
        const int j = idx / WG, col = (idx % WG) * CV;
        C v[CV][R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if constexpr (CV == 1) {
                if (IN_G)
                    v[0][q] = col < wc ? in_g[(size_t)(j + q * nb) * gs + col] : C{T(0), T(0)};
                else
                    v[0][q] = in_s[(j + q * nb) * W + col];
            } else {
                float4 x;
                if (IN_G)
                    x = col < wc ? *reinterpret_cast<const float4 *>(in_g + (size_t)(j + q * nb) * gs + col)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                else
                    x = *reinterpret_cast<const float4 *>(in_s + (j + q * nb) * W + col);
                v[0][q] = C{x.x, x.y};
                v[1][q] = C{x.z, x.w};
            }
        }
        const int jm = j % NS;
        if (NS > 1 && jm != 0) {
#pragma unroll
            for (int q = 1; q < R; ++q) {
                C t = tw[q * jm * step];
                if (sign > 0) t.y = -t.y;
#pragma unroll
                for (int u = 0; u < CV; ++u) v[u][q] = cmul(v[u][q], t);
            }
        }
#pragma unroll
        for (int u = 0; u < CV; ++u) dft<T, C, R>(v[u], sign);
        const int base = (j / NS) * NS * R + jm;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int row = base + q * NS;
            if (MULG && col < wc) {
                const T gv = G[(size_t)row * gstride + (c0 + col) / V];
#pragma unroll
                for (int u = 0; u < CV; ++u) {
                    v[u][q].x *= gv;
                    v[u][q].y *= gv;
                }
            }
            if constexpr (CV == 1) {
                if (OUT_G) {
                    if (col < wc) out_g[(size_t)row * gs + col] = v[0][q];
                } else {
                    out_s[row * W + col] = v[0][q];
                }
            } else {
                const float4 x = make_float4(v[0][q].x, v[0][q].y, v[1][q].x, v[1][q].y);
                if (OUT_G) {
                    if (col < wc) *reinterpret_cast<float4 *>(out_g + (size_t)row * gs + col) = x;
                } else {
                    *reinterpret_cast<float4 *>(out_s + row * W + col) = x;
                }
            }
        }
    }
}

// A run of stages: the first reads the global tile (IN_G) or shared buffer
// sin, intermediate results ping-pong between the shared buffers, the last
// writes the global tile (OUT_G) or shared memory, multiplying by G (MULG).
// Returns the shared buffer holding the result when it stays in shared memory.
template <class T, class C, int K, int W, int NT, int CV, int NS, bool IN_G, bool OUT_G, bool MULG, int R, int... RS>
__device__ __forceinline__ C *ct_pipe(const C *gin, C *gout, size_t gs, int wc, C *sin, C *sout, const C *tw, int sign,
                                      const T *G, size_t gstride, int c0, int V) {
    constexpr bool last = sizeof...(RS) == 0;
    ct_stage<T, C, R, K, W, NT, CV, NS, IN_G, last && OUT_G, last && MULG>(sin, gin, sout, gout, gs, wc, tw, sign, G,
                                                                           gstride, c0, V);
    if constexpr (last) {
        return sout;
    } else {
        __syncthreads();
        return ct_pipe<T, C, K, W, NT, CV, NS * R, false, OUT_G, MULG, RS...>(gin, gout, gs, wc, sout, sin, tw, sign,
                                                                               G, gstride, c0, V);
    }
}

// One 1D pass along the middle axis of [outer][K][inner] (complex) with
// compile-time K, W and radices (at least two stages): a block owns one
// K x W tile.  The first stage loads the global tile straight into registers
// and the last one stores straight from registers, so shared memory carries
// only the exchanges between stages; the fused pass (forward, x G, inverse)
// multiplies by G in the last forward stage.
template <class T, bool FUSED, int K, int W, int NT, int CV, int... RS>
__global__ void __launch_bounds__(NT) k_fft_ct(FFTArgs<T> a) {
    using C = typename Cplx<T>::type;
    static_assert(sizeof...(RS) >= 2, "single-stage sizes would read and write the same global tile");
    extern __shared__ __align__(16) unsigned char smem_ct[];
    C *buf0 = reinterpret_cast<C *>(smem_ct), *buf1 = buf0 + K * W;
    C *tw = buf1 + K * W;
    pdl_launch_dependents();
    for (int i = threadIdx.x; i < K; i += NT) tw[i] = a.tw[i];   // set up once per system
    pdl_wait();
    __syncthreads();
    const int ncb = (a.inner + W - 1) / W;
    const size_t outer = blockIdx.x / ncb;
    const int c0 = (int)(blockIdx.x % ncb) * W;
    const int wc = min(W, a.inner - c0);
    C *base = a.data + outer * (size_t)K * a.inner + c0;
    const size_t gstride = (size_t)(a.inner / a.V);
    if (FUSED) {
        // G of this block's slab: G[outer][row][(c0 + col) / V]
        const T *Gb = a.G + outer * (size_t)K * gstride;
        C *res = ct_pipe<T, C, K, W, NT, CV, 1, true, false, true, RS...>(base, base, a.inner, wc, buf0, buf1, tw,
                                                                           -1, Gb, gstride, c0, a.V);
        __syncthreads();
        C *other = (res == buf0) ? buf1 : buf0;
        ct_pipe<T, C, K, W, NT, CV, 1, false, true, false, RS...>(base, base, a.inner, wc, res, other, tw, +1, a.G,
                                                                   gstride, c0, a.V);
    } else {
        ct_pipe<T, C, K, W, NT, CV, 1, true, true, false, RS...>(base, base, a.inner, wc, buf0, buf1, tw, a.sign,
                                                                  a.G, gstride, c0, a.V);
    }
}

// 16-byte asynchronous copy from global to shared memory (cp.async, cached
// in L2 only), and the group fences of those copies.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit16() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait16() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The same pass over whole tiles with persistent blocks: a block takes tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and, while it transforms one tile
// (from shared memory, last stage written straight to global memory), the
// next tile is already arriving in a second shared buffer by asynchronous
// copies (cp.async, 16 bytes each, issued by all threads).  So the tile loads
// overlap the arithmetic and the stage barriers of the previous tile instead
// of stalling every warp of a block on its own load; the arithmetic per
// element is that of k_fft_ct (bit-identical results).
// Resident blocks of a persistent pass that its shared memory allows (three
// tiles and the twiddles), at most three: the register bound that follows.
template <class T, int K, int W> constexpr int ct_pipe_blocks() {
    constexpr size_t smem = sizeof(typename Cplx<T>::type) * (3 * (size_t)K * W + K) + 1024;
    constexpr size_t per = (227u * 1024u) / smem;
    return per < 1 ? 1 : (per > 3 ? 3 : (int)per);
}

template <class T, bool FUSED, int K, int W, int NT, int CV, int... RS>
__global__ void __launch_bounds__(NT, (ct_pipe_blocks<T, K, W>())) k_fft_ct_pipe(FFTArgs<T> a, unsigned ntiles) {
    using C = typename Cplx<T>::type;
    static_assert(sizeof...(RS) >= 2, "at least two stages");
    static_assert((W * sizeof(C)) % 16 == 0, "tile rows of whole 16-byte chunks");
    constexpr int CPR = (int)(W * sizeof(C) / 16);   // 16-byte chunks per tile row
    constexpr int EPC = (int)(16 / sizeof(C));       // complex values per chunk
    extern __shared__ __align__(16) unsigned char smem_cp[];
    C *in0 = reinterpret_cast<C *>(smem_cp), *in1 = in0 + K * W, *wk = in1 + K * W;
    C *tw = wk + K * W;
    pdl_launch_dependents();
    for (int i = threadIdx.x; i < K; i += NT) tw[i] = a.tw[i];   // set up once per system
    pdl_wait();
    const int ncb = a.inner / W;
    const size_t gstride = (size_t)(a.inner / a.V);
    unsigned t = blockIdx.x;
    if (t < ntiles) {
        const size_t outer = t / ncb;
        const C *src = a.data + outer * (size_t)K * a.inner + (size_t)(t % ncb) * W;
        for (int q = threadIdx.x; q < K * CPR; q += NT)
            cp_async16(in0 + (q / CPR) * W + (q % CPR) * EPC, src + (size_t)(q / CPR) * a.inner + (q % CPR) * EPC);
    }
    cp_async_commit16();
    for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
        C *cur = b ? in1 : in0, *nxt = b ? in0 : in1;
        __syncthreads();                         // every thread is done with nxt (two tiles ago) and wk
        const unsigned tn = t + gridDim.x;
        if (tn < ntiles) {
            const size_t outer = tn / ncb;
            const C *src = a.data + outer * (size_t)K * a.inner + (size_t)(tn % ncb) * W;
            for (int q = threadIdx.x; q < K * CPR; q += NT)
                cp_async16(nxt + (q / CPR) * W + (q % CPR) * EPC,
                           src + (size_t)(q / CPR) * a.inner + (q % CPR) * EPC);
        }
        cp_async_commit16();
        cp_async_wait16<1>();                     // this thread's copies of tile t are done
        __syncthreads();                         // and every thread's
        const size_t outer = t / ncb;
        const int c0 = (int)(t % ncb) * W;
        C *base = a.data + outer * (size_t)K * a.inner + c0;
        if (FUSED) {
            const T *Gb = a.G + outer * (size_t)K * gstride;
            C *res = ct_pipe<T, C, K, W, NT, CV, 1, false, false, true, RS...>(base, base, a.inner, W, cur, wk, tw,
                                                                                -1, Gb, gstride, c0, a.V);
            __syncthreads();
            C *other = (res == cur) ? wk : cur;
            ct_pipe<T, C, K, W, NT, CV, 1, false, true, false, RS...>(base, base, a.inner, W, res, other, tw, +1, Gb,
                                                                       gstride, c0, a.V);
        } else {
            ct_pipe<T, C, K, W, NT, CV, 1, false, true, false, RS...>(base, base, a.inner, W, cur, wk, tw, a.sign,
                                                                       a.G, gstride, c0, a.V);
        }
    }
    cp_async_wait16<0>();                         // no copy in flight at exit
}

template <class T, bool FUSED, int K, int W, int CV, int... RS> int launch_ct_cv(const FFTArgs<T> &a, unsigned grid,
                                                                              cudaStream_t st) {
    using C = typename Cplx<T>::type;
    constexpr int NT = ct_threads<K, W / CV, RS...>();
    if (ct_pipe_blocks<T, K, W>() >= 2 && a.inner % W == 0 && a.sms > 0) {
        // whole tiles and room for two blocks per SM: persistent blocks with the next tile prefetched
        auto kern = k_fft_ct_pipe<T, FUSED, K, W, NT, CV, RS...>;
        const size_t smem = sizeof(C) * (3 * (size_t)K * W + K);
        static int per_sm = -1;                   // resident blocks per SM (one device architecture)
        if (per_sm < 0) {
            int x = 0;
            if (smem > 48 * 1024 &&
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                x = 0;
            else if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, kern, NT, smem) != cudaSuccess)
                x = 0;
            cudaGetLastError();
            per_sm = x;
        }
        if (per_sm > 0) {
            const unsigned pgrid = (unsigned)std::min<long long>(grid, (long long)per_sm * a.sms);
            launch_pdl(a.early != 0, kern, dim3(pgrid), dim3(NT), smem, st, a, grid);
            return 1;
        }
    }
    const size_t smem = sizeof(C) * (2 * (size_t)K * W + K);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_fft_ct<T, FUSED, K, W, NT, CV, RS...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    launch_pdl(a.early != 0, k_fft_ct<T, FUSED, K, W, NT, CV, RS...>, dim3(grid), dim3(NT), smem, st, a);
    return 1;
}

// Float tiles take column pairs when every tile is whole (inner a multiple of
// W), so that the pairs are 16-byte aligned, and V is even, so that the two
// columns of a pair share their G.
template <class T, bool FUSED, int K, int W, int... RS> int launch_ct(const FFTArgs<T> &a, unsigned grid,
                                                                      cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (a.inner % W == 0 && a.V % 2 == 0) return launch_ct_cv<T, FUSED, K, W, 2, RS...>(a, grid, st);
    }
    return launch_ct_cv<T, FUSED, K, W, 1, RS...>(a, grid, st);
}

// The passes of one size: float tiles of 32 or 16 complex columns, double
// tiles of 16.
template <class T, int K, int... RS> int ct_size(const FFTArgs<T> &a, bool fused, unsigned grid, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (a.W == 32) return fused ? launch_ct<T, true, K, 32, RS...>(a, grid, st)
                                    : launch_ct<T, false, K, 32, RS...>(a, grid, st);
        if (a.W == 16) return fused ? launch_ct<T, true, K, 16, RS...>(a, grid, st)
                                    : launch_ct<T, false, K, 16, RS...>(a, grid, st);
    } else {
        if (a.W == 16) return fused ? launch_ct<T, true, K, 16, RS...>(a, grid, st)
                                    : launch_ct<T, false, K, 16, RS...>(a, grid, st);
    }
    return -1;
}

// Spreading fused with the forward FFT along k3: a block owns one (k1, k2)
// pencil of K mesh points and W complex probe-pair columns.  A lane takes CPL
// adjacent columns (CPL = 2: float tiles of 32 columns, one 16-byte dipole
// load per component for four probes), so a warp holds 32 CPL / W row chains.
// The chains spread rows k3 = chain, chain + NSG, ... (two rows per
// iteration: two independent load chains) straight into the shared-memory
// tile, with the records and order of k_spread_csr; then the block transforms
// the tile along k3 and writes it once.  Probe columns >= R are masked to zero.
template <class T, int K, int W, int NT, int CPL, int... RS>
__global__ void __launch_bounds__(NT) k_spread_fft3(const T *__restrict__ d, typename Cplx<T>::type *__restrict__ mesh,
                                                    int R, int ld, int K2, const int *__restrict__ row,
                                                    const SpreadRec<T> *__restrict__ rec,
                                                    const typename Cplx<T>::type *__restrict__ twg) {
    using C = typename Cplx<T>::type;
    constexpr int LPC = W / CPL;              // lanes per row chain
    static_assert(W % CPL == 0 && 32 % LPC == 0, "a warp holds whole row chains");
    static_assert(CPL == 1 || sizeof(T) == 4, "column pairs per lane are float tiles");
    constexpr int G = 32 / LPC;               // row chains per warp
    constexpr int NSG = (NT / 32) * G;        // row chains per block
    constexpr int NP = 2 * CPL;               // probes per lane
    extern __shared__ __align__(16) unsigned char smem_sf[];
    C *buf0 = reinterpret_cast<C *>(smem_sf);
    C *buf1 = buf0 + K * W;
    C *tw = buf1 + K * W;
    pdl_launch_dependents();
    for (int i = threadIdx.x; i < K; i += NT) tw[i] = twg[i];   // set up once per system
    pdl_wait();
    const int V = ld / 2;
    const int ncb = (V + W - 1) / W;
    const size_t pencil = blockIdx.x / ncb;              // k1 * K2 + k2
    const int c0 = (int)(blockIdx.x % ncb) * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = (lane % LPC) * CPL, chain = warp * G + lane / LPC;
    const int col = c0 + cl;                             // complex columns col .. col + CPL - 1 = probes 2 col ..
    const bool on = col < V;
    T msk[NP];
#pragma unroll
    for (int e = 0; e < NP; ++e) msk[e] = (2 * col + e < R) ? T(1) : T(0);
    for (int k3 = chain; k3 < K; k3 += 2 * NSG) {
        const int kb = k3 + NSG;
        const size_t pa = pencil * K + k3, pb = pencil * K + kb;
        int qa = row[pa];
        const int qa1 = row[pa + 1];
        int qb = 0, qb1 = 0;
        if (kb < K) {
            qb = row[pb];
            qb1 = row[pb + 1];
        }
        T acc_a[NP], acc_b[NP];
#pragma unroll
        for (int e = 0; e < NP; ++e) acc_a[e] = acc_b[e] = T(0);
        // the next record of each row is loaded one iteration ahead, so that its
        // latency overlaps the current record's dipole loads
        SpreadRec<T> wa{}, wb{};
        if (qa < qa1) wa = rec[qa];
        if (qb < qb1) wb = rec[qb];
        while (qa < qa1 || qb < qb1) {
            const bool ha = qa < qa1, hb = qb < qb1;
            SpreadRec<T> na = wa, nb = wb;
            if (ha && qa + 1 < qa1) na = rec[qa + 1];
            if (hb && qb + 1 < qb1) nb = rec[qb + 1];
            if (ha) {
                if (on) {
                    T x[NP], y[NP], z[NP];
                    const T *dj = d + (size_t)(3 * wa.atom) * ld + 2 * col;
                    vload<T, NP>(dj, x);
                    vload<T, NP>(dj + ld, y);
                    vload<T, NP>(dj + 2 * (size_t)ld, z);
#pragma unroll
                    for (int e = 0; e < NP; ++e) acc_a[e] += wa.w0 * x[e] + wa.w1 * y[e] + wa.w2 * z[e];
                }
                ++qa;
            }
            if (hb) {
                if (on) {
                    T x[NP], y[NP], z[NP];
                    const T *dj = d + (size_t)(3 * wb.atom) * ld + 2 * col;
                    vload<T, NP>(dj, x);
                    vload<T, NP>(dj + ld, y);
                    vload<T, NP>(dj + 2 * (size_t)ld, z);
#pragma unroll
                    for (int e = 0; e < NP; ++e) acc_b[e] += wb.w0 * x[e] + wb.w1 * y[e] + wb.w2 * z[e];
                }
                ++qb;
            }
            wa = na;
            wb = nb;
        }
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
            buf0[k3 * W + cl + u] = on ? C{acc_a[2 * u] * msk[2 * u], acc_a[2 * u + 1] * msk[2 * u + 1]}
                                       : C{T(0), T(0)};
            if (kb < K)
                buf0[kb * W + cl + u] = on ? C{acc_b[2 * u] * msk[2 * u], acc_b[2 * u + 1] * msk[2 * u + 1]}
                                           : C{T(0), T(0)};
        }
    }
    __syncthreads();
    const int wc = min(W, V - c0);
    C *base = mesh + pencil * (size_t)K * V + c0;
    ct_pipe<T, C, K, W, NT, 1, 1, false, true, false, RS...>(base, base, (size_t)V, wc, buf0, buf1, tw, -1,
                                                              (const T *)nullptr, 0, c0, V);
}

template <class T, int K, int W, int CPL, int... RS>
int launch_sf3_cpl(const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row, const SpreadRec<T> *rec,
                   const typename Cplx<T>::type *tw, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    constexpr int NT = ct_threads<K, W, RS...>();
    const size_t smem = sizeof(C) * (2 * (size_t)K * W + K);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_spread_fft3<T, K, W, NT, CPL, RS...>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    const int V = ld / 2;
    const unsigned grid = (unsigned)((size_t)K1 * K2 * ((V + W - 1) / W));
    launch_pdl(true, k_spread_fft3<T, K, W, NT, CPL, RS...>, dim3(grid), dim3(NT), smem, st, d,
               reinterpret_cast<C *>(mesh), R, ld, K2, row, rec, tw);
    return 1;
}

// Float tiles of 32 columns take two columns per lane when the dipole rows
// allow 16-byte loads (ld a multiple of 4).
template <class T, int K, int W, int... RS>
int launch_sf3(const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row, const SpreadRec<T> *rec,
               const typename Cplx<T>::type *tw, cudaStream_t st) {
    if constexpr (sizeof(T) == 4 && W == 32) {
        if (ld % 4 == 0) return launch_sf3_cpl<T, K, W, 2, RS...>(d, mesh, R, ld, K1, K2, row, rec, tw, st);
    }
    return launch_sf3_cpl<T, K, W, 1, RS...>(d, mesh, R, ld, K1, K2, row, rec, tw, st);
}

template <class T, int K, int... RS>
int sf3_size(int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row, const SpreadRec<T> *rec,
             const typename Cplx<T>::type *tw, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (W == 32) return launch_sf3<T, K, 32, RS...>(d, mesh, R, ld, K1, K2, row, rec, tw, st);
        if (W == 16) return launch_sf3<T, K, 16, RS...>(d, mesh, R, ld, K1, K2, row, rec, tw, st);
    } else {
        if (W == 16) return launch_sf3<T, K, 16, RS...>(d, mesh, R, ld, K1, K2, row, rec, tw, st);
    }
    return -1;
}

// Spreading by pencil records (PencilRec, spline order P) fused with the
// forward FFT along k3: a block owns one (k1, k2) pencil and W complex
// probe-pair columns; lane l holds the PPL = 2W / 32 probes 2 c0 + l PPL ...
// Warp w owns the rows [w K / NW, (w + 1) K / NW) of the pencil.  It walks the
// records of the points (k1, k2, top3) for top3 from its first row to its
// last row + P - 2 (mod K) in CSR order, which is the order of top3, and keeps
// the P rows top3 - P + 1 .. top3 that a record of top3 reaches in registers:
// each record adds M3(t3) (e0 . d_j) + M3'(t3) (e1 . d_j) to row top3 - t3.
// When top3 moves past a row's last contributor the row is complete and goes
// to the shared tile (rows outside the warp's range belong to a neighbour and
// are dropped), so every row is a sum in a fixed order.  The next record is
// loaded one iteration ahead.  The block then transforms the tile along k3 and
// writes it once.  Probes >= R are zero.
template <class T, int K, int W, int NT, int P, int... RS>
__global__ void __launch_bounds__(NT) k_spread_pencil_fft3(const T *__restrict__ d,
                                                           typename Cplx<T>::type *__restrict__ mesh, int R, int ld,
                                                           const int *__restrict__ prow,
                                                           const PencilRec<T> *__restrict__ prec,
                                                           const T *__restrict__ k3w,
                                                           const typename Cplx<T>::type *__restrict__ twg) {
    using C = typename Cplx<T>::type;
    constexpr int PPL = 2 * W / 32;           // probes per lane
    static_assert(PPL == 1 || PPL == 2, "tiles of 16 or 32 complex columns");
    static_assert(P <= 8, "k3 stencils hold at most 8 points");
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_spp[];
    C *buf0 = reinterpret_cast<C *>(smem_spp);
    C *buf1 = buf0 + K * W;
    C *tw = buf1 + K * W;
    int *rp = reinterpret_cast<int *>(tw + K);   // [K + 1] record starts of the pencil's points
    pdl_launch_dependents();
    const int V = ld / 2;
    const int ncb = V / W;
    const size_t pencil = blockIdx.x / ncb;      // k1 * K2 + k2
    const int c0 = (int)(blockIdx.x % ncb) * W;
    for (int i = threadIdx.x; i < K; i += NT) tw[i] = twg[i];   // set up once per system
    for (int i = threadIdx.x; i <= K; i += NT) rp[i] = prow[pencil * K + i];
    pdl_wait();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = warp * K / NW, r1 = (warp + 1) * K / NW;
    const int pr0 = 2 * c0 + lane * PPL;        // first probe of the lane
    T msk[PPL];
#pragma unroll
    for (int e = 0; e < PPL; ++e) msk[e] = pr0 + e < R ? T(1) : T(0);
    T *tile = reinterpret_cast<T *>(buf0);      // [K][2W] reals
    T acc[P][PPL];                              // acc[j]: row cur - P + 1 + j
#pragma unroll
    for (int j = 0; j < P; ++j)
#pragma unroll
        for (int e = 0; e < PPL; ++e) acc[j][e] = T(0);
    int cur = r0;
    // row cur - P + 1 is complete: to the tile if it is this warp's, then shift the window
#define MBD_SPP_FLUSH_ADVANCE()                                                                     \
    do {                                                                                            \
        const int row_ = cur - P + 1;                                                               \
        if (row_ >= r0) {                                                                           \
            _Pragma("unroll") for (int e = 0; e < PPL; ++e) tile[row_ * 2 * W + lane * PPL + e] =   \
                acc[0][e] * msk[e];                                                                 \
        }                                                                                           \
        _Pragma("unroll") for (int j = 0; j < P - 1; ++j)                                          \
            _Pragma("unroll") for (int e = 0; e < PPL; ++e) acc[j][e] = acc[j + 1][e];             \
        _Pragma("unroll") for (int e = 0; e < PPL; ++e) acc[P - 1][e] = T(0);                      \
        ++cur;                                                                                      \
    } while (0)
    // the last (unwrapped) top3 reaching row r1 - 1; beyond K it wraps to 0..
    const int last = r1 + P - 2;
    for (int seg = 0; seg < 2; ++seg) {
        const int t_lo = seg == 0 ? r0 : K, t_hi = seg == 0 ? min(last, K - 1) : last;   // top3 (+ K) range
        if (t_hi < t_lo) continue;
        int q = rp[t_lo - seg * K];
        const int qe = rp[t_hi - seg * K + 1];
        PencilRec<T> rc{};
        if (q < qe) rc = prec[q];
        for (; q < qe; ++q) {
            PencilRec<T> rn = rc;
            if (q + 1 < qe) rn = prec[q + 1];
            T x[PPL], y[PPL], z[PPL];
            const T *dj = d + (size_t)(3 * rc.atom) * ld + pr0;
            vload<T, PPL>(dj, x);
            vload<T, PPL>(dj + ld, y);
            vload<T, PPL>(dj + 2 * (size_t)ld, z);
            T m3[P], n3[P];
            {
                // the atom's row of 16 values (M3 at 0.., M3' at 8..), 16-byte loads
                constexpr int U = 16 / (int)sizeof(T);
                const T *kw = k3w + (size_t)rc.atom * 16;
                T row[16];
#pragma unroll
                for (int b = 0; b < 16; b += U) {
                    if (b < P || (b + U > 8 && b < 8 + P)) vload<T, U>(kw + b, row + b);
                }
#pragma unroll
                for (int t = 0; t < P; ++t) {
                    m3[t] = row[t];
                    n3[t] = row[8 + t];
                }
            }
            // complete the rows no record of this top3 or later reaches
            const int tcur = rc.top3 + seg * K;
            while (cur < tcur) MBD_SPP_FLUSH_ADVANCE();
#pragma unroll
            for (int e = 0; e < PPL; ++e) {
                const T u = rc.e0[0] * x[e] + rc.e0[1] * y[e] + rc.e0[2] * z[e];
                const T v = rc.e1[0] * x[e] + rc.e1[1] * y[e] + rc.e1[2] * z[e];
#pragma unroll
                for (int t = 0; t < P; ++t) acc[P - 1 - t][e] += m3[t] * u + n3[t] * v;
            }
            rc = rn;
        }
    }
    while (cur <= last) MBD_SPP_FLUSH_ADVANCE();
#undef MBD_SPP_FLUSH_ADVANCE
    __syncthreads();
    // the forward k3 transform of the whole tile; float tiles take column
    // pairs (one 16-byte access and one twiddle for two columns)
    C *base = mesh + pencil * (size_t)K * V + c0;
    constexpr int CV = sizeof(T) == 4 ? 2 : 1;
    ct_pipe<T, C, K, W, NT, CV, 1, false, true, false, RS...>(base, base, (size_t)V, W, buf0, buf1, tw, -1,
                                                               (const T *)nullptr, 0, c0, V);
}

template <class T, int K, int W, int... RS>
int launch_spp(const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow, const PencilRec<T> *prec,
               const T *k3w, const typename Cplx<T>::type *tw, cudaStream_t st) {
    using C = typename Cplx<T>::type;
    constexpr int NT = ct_threads<K, W, RS...>();
    static_assert(NT % 32 == 0 && K >= 2 * 6, "whole warps; K >= 2p");
    const size_t smem = sizeof(C) * (2 * (size_t)K * W + K) + sizeof(int) * (K + 1);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_spread_pencil_fft3<T, K, W, NT, 6, RS...>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    const int V = ld / 2;
    const unsigned grid = (unsigned)((size_t)K1 * K2 * (V / W));
    launch_pdl(true, k_spread_pencil_fft3<T, K, W, NT, 6, RS...>, dim3(grid), dim3(NT), smem, st, d,
               reinterpret_cast<C *>(mesh), R, ld, prow, prec, k3w, tw);
    return 1;
}

template <class T, int K, int... RS>
int spp_size(int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow, const PencilRec<T> *prec,
             const T *k3w, const typename Cplx<T>::type *tw, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (W == 32) return launch_spp<T, K, 32, RS...>(d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st);
        if (W == 16) return launch_spp<T, K, 16, RS...>(d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st);
    } else {
        if (W == 16) return launch_spp<T, K, 16, RS...>(d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st);
    }
    return -1;
}

}  // namespace

// The translation unit of group g: dispatch over its sizes.
#define MBD_CT_CASE(K, ...) \
    case K: return ct_size<T, K, __VA_ARGS__>(a, fused, grid, st);
#define MBD_SF3_CASE(K, ...) \
    case K: return sf3_size<T, K, __VA_ARGS__>(W, d, mesh, R, ld, K1, K2, row, rec, tw, st);
#define MBD_SPP_CASE(K, ...) \
    case K: return spp_size<T, K, __VA_ARGS__>(W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st);
#define MBD_FFT_GROUP_TU(g)                                                                                       \
    template <class T> int launch_fft_ct_group##g(const FFTArgs<T> &a, bool fused, unsigned grid, cudaStream_t st) { \
        switch (a.K) { MBD_FFT_GROUP##g(MBD_CT_CASE) default: return -1; }                                         \
    }                                                                                                              \
    template <class T>                                                                                             \
    int launch_sf3_group##g(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row,    \
                            const SpreadRec<T> *rec, const typename Cplx<T>::type *tw, cudaStream_t st) {          \
        switch (K3) { MBD_FFT_GROUP##g(MBD_SF3_CASE) default: return -1; }                                         \
    }                                                                                                              \
    template int launch_fft_ct_group##g<float>(const FFTArgs<float> &, bool, unsigned, cudaStream_t);              \
    template int launch_fft_ct_group##g<double>(const FFTArgs<double> &, bool, unsigned, cudaStream_t);            \
    template int launch_sf3_group##g<float>(int, int, const float *, float *, int, int, int, int, const int *,     \
                                            const SpreadRec<float> *, const float2 *, cudaStream_t);               \
    template int launch_sf3_group##g<double>(int, int, const double *, double *, int, int, int, int, const int *,  \
                                             const SpreadRec<double> *, const double2 *, cudaStream_t);           \
    template <class T>                                                                                             \
    int launch_spp_group##g(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow,    \
                            const PencilRec<T> *prec, const T *k3w, const typename Cplx<T>::type *tw,              \
                            cudaStream_t st) {                                                                     \
        switch (K3) { MBD_FFT_GROUP##g(MBD_SPP_CASE) default: return -1; }                                         \
    }                                                                                                              \
    template int launch_spp_group##g<float>(int, int, const float *, float *, int, int, int, int, const int *,     \
                                            const PencilRec<float> *, const float *, const float2 *, cudaStream_t); \
    template int launch_spp_group##g<double>(int, int, const double *, double *, int, int, int, int, const int *,  \
                                             const PencilRec<double> *, const double *, const double2 *,          \
                                             cudaStream_t);

}  // namespace mbd
