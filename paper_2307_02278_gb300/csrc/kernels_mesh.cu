// Per-step operator kernels: SPME spreading (Eq. dipolarr), the batched 3D FFT
// convolution with the influence function (Eq. spme), and the fused field
// kernel (SPME gather + real-space pairs + self term, Eqs. spme, fld_ewald,
// fld_ewald1) with the Lanczos epilogue l_k = Omega y_k + Diag(g) E*_k and
// a_k = y_k^T l_k (Eqs. lk3, recurs2).
#include "fft.cuh"

#include <algorithm>

namespace mbd {

namespace {

constexpr int kWarps = 8;          // warps per block in the field kernel

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

// The same rows with a block per brick: the candidate atoms of the brick's
// points (the atoms of its nc1 x nc2 x nc3 candidate bricks, in the order the
// per-point kernel visits them) are staged once in shared memory, with their
// top stencil points, and a thread per point of the brick tests them there.
// The rows are identical to k_spread_rows'.  A brick with more than
// kRowsCap candidates reads them from global memory instead.
constexpr int kRowsCap = 512;
constexpr int kRowsMaxBins = 512;
template <class T, bool FILL>
__global__ void k_spread_rows_brick(Geom g, BinView B, const int *__restrict__ top, const double *__restrict__ w64,
                                    const double *__restrict__ dw64, int *__restrict__ cnt_or_row,
                                    SpreadRec<T> *__restrict__ rec) {
    __shared__ int cj[kRowsCap], ct[kRowsCap][3];
    __shared__ int boff[kRowsMaxBins + 1], bfirst[kRowsMaxBins];
    const int tid = threadIdx.x;
    const int brick = blockIdx.x;
    const int bb1 = brick / (B.nb2 * B.nb3), bb2 = (brick / B.nb3) % B.nb2, bb3 = brick % B.nb3;
    const int nbc = B.nc1 * B.nc2 * B.nc3;
    for (int t = tid; t < nbc; t += blockDim.x) {
        const int c1 = t / (B.nc2 * B.nc3), c2 = (t / B.nc3) % B.nc2, c3 = t % B.nc3;
        const int bin = (((bb1 + c1) % B.nb1) * B.nb2 + (bb2 + c2) % B.nb2) * B.nb3 + (bb3 + c3) % B.nb3;
        bfirst[t] = B.start[bin];
        boff[t + 1] = B.start[bin + 1] - B.start[bin];
    }
    __syncthreads();
    if (tid == 0) {
        boff[0] = 0;
        for (int t = 0; t < nbc; ++t) boff[t + 1] += boff[t];
    }
    __syncthreads();
    const int total = boff[nbc];
    const bool staged = total <= kRowsCap;
    if (staged) {
        for (int k = tid; k < total; k += blockDim.x) {
            int lo = 0, hi = nbc - 1;   // the candidate brick holding entry k
            while (lo < hi) {
                const int mid = (lo + hi + 1) / 2;
                if (boff[mid] <= k) lo = mid;
                else hi = mid - 1;
            }
            const int j = B.atoms[bfirst[lo] + (k - boff[lo])];
            cj[k] = j;
            ct[k][0] = top[3 * j];
            ct[k][1] = top[3 * j + 1];
            ct[k][2] = top[3 * j + 2];
        }
    }
    __syncthreads();
    const int npb = B.bs1 * B.bs2 * B.bs3;
    if (tid >= npb) return;
    const int g1 = bb1 * B.bs1 + tid / (B.bs2 * B.bs3), g2 = bb2 * B.bs2 + (tid / B.bs3) % B.bs2,
              g3 = bb3 * B.bs3 + tid % B.bs3;
    const size_t pt = ((size_t)g1 * g.K2 + g2) * g.K3 + g3;
    const int p = g.p;
    int c = 0;
    const int base = FILL ? cnt_or_row[pt] : 0;
    for (int k = 0; k < total; ++k) {
        int j, tj1, tj2, tj3;
        if (staged) {
            j = cj[k];
            tj1 = ct[k][0];
            tj2 = ct[k][1];
            tj3 = ct[k][2];
        } else {
            int t = 0;
            while (boff[t + 1] <= k) ++t;
            j = B.atoms[bfirst[t] + (k - boff[t])];
            tj1 = top[3 * j];
            tj2 = top[3 * j + 1];
            tj3 = top[3 * j + 2];
        }
        int u1 = tj1 - g1;
        if (u1 < 0) u1 += g.K1;
        int u2 = tj2 - g2;
        if (u2 < 0) u2 += g.K2;
        int u3 = tj3 - g3;
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
    if (!FILL) cnt_or_row[pt] = c;
}

// Pencil records (PencilRec): a thread per mesh point (k1, k2, k3) finds the
// atoms whose top stencil point is (k1 + t1, k2 + t2, k3), t1, t2 < p (mod K),
// in the bricks that hold those tops, visited in a fixed order (candidate
// bricks in order, atoms of a brick by index), so the records of a point come
// in a fixed order.  FILL = false counts, FILL = true writes e0 and e1 from
// the FP64 stencil weights.
template <class T, bool FILL>
__global__ void k_pencil_rows(Geom g, BinView B, const int *__restrict__ top, const double *__restrict__ w64,
                              const double *__restrict__ dw64, int *__restrict__ cnt_or_row,
                              PencilRec<T> *__restrict__ rec) {
    const size_t npts = (size_t)g.K1 * g.K2 * g.K3;
    const size_t pt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pt >= npts) return;
    const int g3 = (int)(pt % g.K3), g2 = (int)((pt / g.K3) % g.K2), g1 = (int)(pt / ((size_t)g.K2 * g.K3));
    const int p = g.p;
    // bricks holding tops in [g1, g1 + p - 1] (and likewise along k2), the one holding k3
    const int b1 = g1 / B.bs1, b2 = g2 / B.bs2, b3 = g3 / B.bs3;
    const int n1 = min(B.nb1, (g1 + p - 1) / B.bs1 - b1 + 1);
    const int n2 = min(B.nb2, (g2 + p - 1) / B.bs2 - b2 + 1);
    int c = 0;
    const int base = FILL ? cnt_or_row[pt] : 0;
    for (int c1 = 0; c1 < n1; ++c1) {
        const int t1b = (b1 + c1) % B.nb1;
        for (int c2 = 0; c2 < n2; ++c2) {
            const int t2b = (b2 + c2) % B.nb2;
            const int bin = (t1b * B.nb2 + t2b) * B.nb3 + b3;
            for (int s = B.start[bin]; s < B.start[bin + 1]; ++s) {
                const int j = B.atoms[s];
                if (top[3 * j + 2] != g3) continue;
                int u1 = top[3 * j] - g1;
                if (u1 < 0) u1 += g.K1;
                int u2 = top[3 * j + 1] - g2;
                if (u2 < 0) u2 += g.K2;
                if (u1 >= p || u2 >= p) continue;
                if (FILL) {
                    const double *w = w64 + (size_t)3 * p * j, *dw = dw64 + (size_t)3 * p * j;
                    const double m1 = w[u1], m2 = w[p + u2], n1v = dw[u1], n2v = dw[p + u2];
                    const double a = n1v * m2, b = m1 * n2v, cc = m1 * m2;
                    PencilRec<T> r;
#pragma unroll
                    for (int al = 0; al < 3; ++al) {
                        r.e0[al] = T(g.cmat[al] * a + g.cmat[3 + al] * b);
                        r.e1[al] = T(g.cmat[6 + al] * cc);
                    }
                    r.atom = j;
                    r.top3 = g3;
                    rec[base + c] = r;
                }
                ++c;
            }
        }
    }
    if (!FILL) cnt_or_row[pt] = c;
}

// The k3 stencil of each atom for the pencil spreading: k3w[j][t] = M3(t),
// k3w[j][8 + t] = M3'(t) (t < p <= 8), zero elsewhere.
template <class T>
__global__ void k_pencil_k3w(int N, int p, const double *__restrict__ w64, const double *__restrict__ dw64,
                             T *__restrict__ k3w) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 16 * N) return;
    const int j = idx / 16, t = idx % 16;
    const int tt = t & 7;
    double v = 0.0;
    if (tt < p) v = (t < 8 ? w64 : dw64)[(size_t)(3 * j + 2) * p + tt];
    k3w[idx] = T(v);
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
        // G index: (outer, row, (c0 + col) / V)
        const T *Gb = a.G + outer * (size_t)a.K * (a.inner / a.V);
        for (int idx = threadIdx.x; idx < a.K * a.W; idx += blockDim.x) {
            const int row = idx / a.W, col = idx - row * a.W;
            if (col < wc) {
                const T gv = Gb[(size_t)row * (a.inner / a.V) + (c0 + col) / a.V];
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

// ---------------------------------------------------------------- real space on clusters
template <class T> struct RealArgs {
    const T *d;          // [N][3][ld]
    T *out;              // [N][3][ld] E_real
    int ld, N, nclus;
    const int *order;    // cluster c = atoms order[16c .. 16c + 15]
    const int *estart;   // [nclus + 1] entry starts
    const int *pstart;   // [16 nclus + 1] pair starts per (cluster, atom)
    const int *entries;  // distinct neighbours j of each cluster
    const RealPair<T> *pairs;
};

// The real-space field E_real = sum over pairs A(r) d_j (Eq. fld_ewald with
// the damping correction) on clusters: a block per cluster of 16 atoms and
// probe chunk (blockIdx.y, 32 PPL probes), warp w for cluster atom w, lanes
// over PPL consecutive probes.  The block stages the dipoles of the cluster's
// distinct neighbours in shared memory, kRealCE entries at a time (coalesced
// 16-byte loads by all threads), so each neighbour's dipoles come from L2
// once per cluster.  Each warp reads its atom's pairs (entry index and
// tensor) 32 at a time into shared memory, one per lane, counts by a ballot
// those whose entries are staged (entries increase along a batch) and applies
// them with no test per pair, accumulating in registers: no global load waits
// inside the pair loop.  An atom's field is the sum over its pairs in
// (j, image) order: deterministic.
constexpr int kRealCE = 48;
template <class T, int PPL>
__global__ void __launch_bounds__(32 * kClusterSize) k_real_clusters(RealArgs<T> a) {
    constexpr int NP = 32 * PPL;                   // probes of the block
    constexpr int U = 16 / (int)sizeof(T);         // values per 16-byte load
    constexpr int PER_ROW = NP / U;                // 16-byte loads per staged row
    // dynamic shared memory: the staged dipoles [kRealCE][3][NP], then the
    // warps' batches of pairs [kClusterSize][32]
    extern __shared__ __align__(16) unsigned char real_smem[];
    T(*sd)[3][NP] = reinterpret_cast<T(*)[3][NP]>(real_smem);
    RealPair<T>(*sp)[32] = reinterpret_cast<RealPair<T>(*)[32]>(real_smem + sizeof(T) * kRealCE * 3 * NP);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x;
    const int pb = blockIdx.y * NP;
    const int r0 = pb + lane * PPL;
    const bool inld = r0 < a.ld;
    const bool vec = a.ld % U == 0;
    const int eb = a.estart[c], ee = a.estart[c + 1];
    const int slot = c * kClusterSize + warp;
    const int pe = a.pstart[slot + 1];
    int bbase = a.pstart[slot], bn = 0, bi = 0;    // the warp's batch of pairs [bbase, bbase + bn), next bi
    int ev = 0x7fffffff;                           // entry of the batch's pair held by this lane
    T E[3][PPL];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int e = 0; e < PPL; ++e) E[k][e] = T(0);
    for (int c0 = eb; c0 < ee; c0 += kRealCE) {
        const int ne = min(kRealCE, ee - c0);
        __syncthreads();                           // the previous chunk is consumed
        for (int t = threadIdx.x; t < ne * 3 * PER_ROW; t += blockDim.x) {
            const int q = t / (3 * PER_ROW), rem = t - q * (3 * PER_ROW), k = rem / PER_ROW, u = rem - k * PER_ROW;
            const T *src = a.d + (size_t)(3 * a.entries[c0 + q] + k) * a.ld + pb + u * U;
            T *dst = &sd[q][k][u * U];
            if (vec && pb + u * U + U <= a.ld) {
                *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(src);
            } else {
#pragma unroll
                for (int v = 0; v < U; ++v) dst[v] = pb + u * U + v < a.ld ? src[v] : T(0);
            }
        }
        __syncthreads();
        const int lo = c0 - eb, lim = lo + ne;     // entries staged: [lo, lim)
        for (;;) {
            if (bi == bn) {                        // the next 32 pairs of this atom
                bbase += bn;
                if (bbase >= pe) break;
                bn = min(32, pe - bbase);
                bi = 0;
                __syncwarp();
                if (lane < bn) {
                    const RealPair<T> r = a.pairs[bbase + lane];
                    sp[warp][lane] = r;
                    ev = r.e;
                } else {
                    ev = 0x7fffffff;
                }
                __syncwarp();
            }
            // the pairs bi .. bi + cnt - 1 of the batch have their entries staged
            // (entries increase along the batch)
            const int cnt = __popc(__ballot_sync(0xffffffffu, lane >= bi && ev < lim));
            for (int t = 0; t < cnt; ++t) {
                const RealPair<T> &cur = sp[warp][bi + t];
                const int q = cur.e - lo;
                T x[PPL], y[PPL], z[PPL];
                vload<T, PPL>(&sd[q][0][lane * PPL], x);
                vload<T, PPL>(&sd[q][1][lane * PPL], y);
                vload<T, PPL>(&sd[q][2][lane * PPL], z);
                const T A0 = cur.a[0], A1 = cur.a[1], A2 = cur.a[2], A3 = cur.a[3], A4 = cur.a[4], A5 = cur.a[5];
#pragma unroll
                for (int e = 0; e < PPL; ++e) {
                    E[0][e] += A0 * x[e] + A1 * y[e] + A2 * z[e];
                    E[1][e] += A1 * x[e] + A3 * y[e] + A4 * z[e];
                    E[2][e] += A2 * x[e] + A4 * y[e] + A5 * z[e];
                }
            }
            bi += cnt;
            if (bi < bn) break;                    // the next pair waits for a later chunk
        }
    }
    const int idx = c * kClusterSize + warp;
    if (!inld || idx >= a.N) return;
    const int i = a.order[idx];
#pragma unroll
    for (int k = 0; k < 3; ++k) vstore<T, PPL>(a.out + (size_t)(3 * i + k) * a.ld + r0, E[k]);
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
    const T *ereal;      // when set: the real-space field from k_real_clusters [N][3][ld]
    FieldOut<T> o;
};

// Field kernel: one block works on `apb` atoms in turn; for each atom its NW
// warps split the work (warp w takes stencil planes t1 = w, w + NW, ... and,
// with the pair loop, neighbours nb0 + w, nb0 + w + NW, ...; warp 0 adds the
// self term, warp NW - 1 the real-space field of the clusters), lanes own VEC
// consecutive probes.  NW = 8, or NW = p = 6 when the real space comes from
// the clusters (one warp per stencil plane, none idle).  The 8 partial fields are summed in a fixed order in
// shared memory and the epilogue selected by o.mode runs with one thread per
// probe: E* = E^rec + E^dir + E^self (Eqs. ewalddip, spme, fld_ewald,
// fld_ewald1), l_k = Omega y_k + Diag(g) E*_k and a_k = y_k^T l_k (Eqs. lk3,
// recurs2).  PC = spline order (0: runtime).
template <class T, int VEC, int PC, int NW, int LPA = 32>
__global__ void __launch_bounds__(NW * 32, NW == kWarps ? ((VEC <= 2 && sizeof(T) == 4 && PC > 0) ? 3 : 2)
                                                        : (LPA == 16 ? 4 : ((VEC <= 2 && sizeof(T) == 4) ? 4 : 2)))
    k_field(FieldArgs<T> a, int apb) {
    // atoms per iteration: with six warps (no pair loop) and four probes per
    // lane, two atoms are gathered together, their loads interleaved, sharing
    // one barrier (128 probes: 585 -> 527 us per launch at 128^3); with
    // fewer probes per lane the registers this takes cost a resident block
    // (64 probes at 192^3: 1236 -> 1369 us).  LPA = 16 (six warps, 64-probe
    // chunks, four probes per lane): each half-warp gathers its own atom, so a
    // warp takes two atoms with one atom's registers per lane.
    constexpr bool HALF = LPA == 16;
    static_assert(!HALF || (NW != kWarps && VEC == 4), "half-warp atoms: six warps, four probes per lane");
    constexpr int AIT = HALF ? 2 : ((NW != kWarps && VEC == 4) ? 2 : 1);   // atoms per iteration
    constexpr int APT = HALF ? 1 : AIT;                                    // atoms per lane
    constexpr int NLOC = LPA * VEC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = HALF ? (lane >> 4) : 0;          // the lane's atom of the iteration (half-warp mode)
    const int lid = HALF ? (lane & 15) : lane;
    const int rbase = blockIdx.y * NLOC;
    const int r0 = rbase + lid * VEC;
    const bool inld = r0 < a.ld;
    const int p = PC > 0 ? PC : a.g.p;
    // partial fields of the warps, double-buffered by atom iteration: the
    // barrier after one iteration's writes also orders the previous epilogue's
    // reads before the buffer is written again, so one barrier per iteration
    __shared__ T red[2][AIT][NW][3][NLOC];
    __shared__ double bsum[NLOC];
    __shared__ double pcarry[3 * NLOC > NW * 32 ? 3 * NLOC - NW * 32 : 1];
    __shared__ double pall[3 * NLOC];
    pdl_launch_dependents();
    for (int k = threadIdx.x; k < (3 * NLOC > NW * 32 ? 3 * NLOC - NW * 32 : 1); k += blockDim.x)
        pcarry[k] = 0.0;
    pdl_wait();
    double part = 0.0;                          // y.l of the (component, probe) this thread owns
    for (int ai = 0; ai < apb; ai += AIT) {
        const int rb = (ai / AIT) & 1;
        int iat[AIT];
        bool val[AIT];
#pragma unroll
        for (int aa = 0; aa < AIT; ++aa) {
            const int idx = blockIdx.x * apb + ai + aa;
            val[aa] = ai + aa < apb && idx < a.g.N;
            iat[aa] = val[aa] ? a.order[idx] : 0;
        }
        if (!val[0]) break;
        // the lane's own atom in half-warp mode (a select, not an indexed array)
        const int my_i = (HALF && sub) ? iat[AIT - 1] : iat[0];
        const bool my_v = (HALF && sub) ? val[AIT - 1] : val[0];
        T E0[APT][VEC], E1[APT][VEC], E2[APT][VEC];
#pragma unroll
        for (int aa = 0; aa < APT; ++aa)
#pragma unroll
            for (int v = 0; v < VEC; ++v) E0[aa][v] = E1[aa][v] = E2[aa][v] = T(0);
        if (inld) {
            if (a.o.terms & MBD_TERM_RECIP) {
                T f0[APT][VEC], f1[APT][VEC], f2[APT][VEC];
                int top1[APT], top2[APT], top3[APT];
                const T *w[APT], *dw[APT];
#pragma unroll
                for (int aa = 0; aa < APT; ++aa) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) f0[aa][v] = f1[aa][v] = f2[aa][v] = T(0);
                    const int i = HALF ? my_i : iat[aa];
                    top1[aa] = a.sp.top[3 * i];
                    top2[aa] = a.sp.top[3 * i + 1];
                    top3[aa] = a.sp.top[3 * i + 2];
                    w[aa] = a.sp.w + (size_t)3 * p * i;
                    dw[aa] = a.sp.dw + (size_t)3 * p * i;
                }
                for (int t1 = warp; t1 < p; t1 += NW) {
                    int k1[APT];
                    T wa[APT], da[APT];
#pragma unroll
                    for (int aa = 0; aa < APT; ++aa) {
                        k1[aa] = top1[aa] - t1;
                        if (k1[aa] < 0) k1[aa] += a.g.K1;
                        wa[aa] = w[aa][t1];
                        da[aa] = dw[aa][t1];
                    }
#pragma unroll
                    for (int t2 = 0; t2 < (PC > 0 ? PC : kMaxOrder); ++t2) {
                        if (t2 >= p) break;
                        const T *rowp[APT];
                        T ab[APT], Ab[APT], aB[APT];
#pragma unroll
                        for (int aa = 0; aa < APT; ++aa) {
                            int k2 = top2[aa] - t2;
                            if (k2 < 0) k2 += a.g.K2;
                            const T wb = w[aa][p + t2], db = dw[aa][p + t2];
                            ab[aa] = wa[aa] * wb;
                            Ab[aa] = da[aa] * wb;
                            aB[aa] = wa[aa] * db;
                            rowp[aa] = a.mesh + ((size_t)k1[aa] * a.g.K2 + k2) * a.g.K3 * a.ld + r0;
                        }
#pragma unroll
                        for (int t3 = 0; t3 < (PC > 0 ? PC : kMaxOrder); ++t3) {
                            if (t3 >= p) break;
                            T phi[APT][VEC];
#pragma unroll
                            for (int aa = 0; aa < APT; ++aa) {
                                int k3 = top3[aa] - t3;
                                if (k3 < 0) k3 += a.g.K3;
                                vload<T, VEC>(rowp[aa] + (size_t)k3 * a.ld, phi[aa]);
                            }
#pragma unroll
                            for (int aa = 0; aa < APT; ++aa) {
                                const T wc = w[aa][2 * p + t3], dc = dw[aa][2 * p + t3];
                                const T c0 = Ab[aa] * wc, c1 = aB[aa] * wc, c2 = ab[aa] * dc;
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    f0[aa][v] += c0 * phi[aa][v];
                                    f1[aa][v] += c1 * phi[aa][v];
                                    f2[aa][v] += c2 * phi[aa][v];
                                }
                            }
                        }
                    }
                }
                // E^rec_alpha = sum_beta C_{beta alpha} f_beta
                const T m00 = T(a.g.cmat[0]), m01 = T(a.g.cmat[1]), m02 = T(a.g.cmat[2]);
                const T m10 = T(a.g.cmat[3]), m11 = T(a.g.cmat[4]), m12 = T(a.g.cmat[5]);
                const T m20 = T(a.g.cmat[6]), m21 = T(a.g.cmat[7]), m22 = T(a.g.cmat[8]);
#pragma unroll
                for (int aa = 0; aa < APT; ++aa)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        E0[aa][v] += m00 * f0[aa][v] + m10 * f1[aa][v] + m20 * f2[aa][v];
                        E1[aa][v] += m01 * f0[aa][v] + m11 * f1[aa][v] + m21 * f2[aa][v];
                        E2[aa][v] += m02 * f0[aa][v] + m12 * f1[aa][v] + m22 * f2[aa][v];
                    }
            }
#pragma unroll
            for (int aa = 0; aa < APT; ++aa) {
                if (!(HALF ? my_v : val[aa])) continue;
                const int i = HALF ? my_i : iat[aa];
                if ((a.o.terms & MBD_TERM_REAL) && a.ereal != nullptr) {
                    if (warp == NW - 1) {
                        T x[VEC], y[VEC], z[VEC];
                        const T *ei = a.ereal + (size_t)(3 * i) * a.ld + r0;
                        vload<T, VEC>(ei, x);
                        vload<T, VEC>(ei + a.ld, y);
                        vload<T, VEC>(ei + 2 * (size_t)a.ld, z);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            E0[aa][v] += x[v];
                            E1[aa][v] += y[v];
                            E2[aa][v] += z[v];
                        }
                    }
                } else if (!HALF && (a.o.terms & MBD_TERM_REAL)) {
                    const int nb1 = a.pr.row[i + 1];
                    constexpr int B4 = 4;
                    for (int nb = a.pr.row[i] + warp; nb < nb1; nb += B4 * NW) {
                        int jj[B4];
#pragma unroll
                        for (int u = 0; u < B4; ++u) jj[u] = (nb + u * NW < nb1) ? a.pr.col[nb + u * NW] : -1;
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
                                const T *A = a.pr.A + 6 * (size_t)(nb + u * NW);
                                const T A0 = A[0], A1 = A[1], A2 = A[2], A3 = A[3], A4 = A[4], A5 = A[5];
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    E0[aa][v] += A0 * xs[u][v] + A1 * ys[u][v] + A2 * zs[u][v];
                                    E1[aa][v] += A1 * xs[u][v] + A3 * ys[u][v] + A4 * zs[u][v];
                                    E2[aa][v] += A2 * xs[u][v] + A4 * ys[u][v] + A5 * zs[u][v];
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
                        E0[aa][v] += c * x[v];
                        E1[aa][v] += c * y[v];
                        E2[aa][v] += c * z[v];
                    }
                }
            }
        }
#pragma unroll
        for (int aa = 0; aa < APT; ++aa)
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                red[rb][HALF ? sub : aa][warp][0][lid * VEC + v] = E0[aa][v];
                red[rb][HALF ? sub : aa][warp][1][lid * VEC + v] = E1[aa][v];
                red[rb][HALF ? sub : aa][warp][2][lid * VEC + v] = E2[aa][v];
            }
        __syncthreads();
        // epilogue: one thread per (component, probe) so that the FP64 work
        // spreads over the warps; the atoms of the iteration in order
#pragma unroll
        for (int aa = 0; aa < AIT; ++aa) {
            if (!val[aa]) continue;
            const int i = iat[aa];
            for (int cp = threadIdx.x; cp < 3 * NLOC; cp += blockDim.x) {
                const int c = cp / NLOC, t = cp - c * NLOC;
                const int r = rbase + t;
                if (r < a.ld) {
                    T sum = T(0);
#pragma unroll
                    for (int w = 0; w < NW; ++w) sum += red[rb][aa][w][c][t];
                    const double E = double(sum);
                    const size_t o = (size_t)(3 * i + c) * a.ld + r;
                    if (a.o.mode == kFieldOut) {
                        a.o.out[o] = E;
                    } else if (a.o.mode == kFieldApply) {
                        a.o.out[o] = a.w2[i] * a.o.xin[o] + a.g_at[i] * E;
                    } else {
                        const double invb = a.o.lz.invb[r];
                        double *Yk = a.o.lz.Y + lz_slot(a.o.lz, a.o.k) * (size_t)(3 * a.g.N) * a.ld;
                        const double y = Yk[o] * invb;
                        const double l = a.w2[i] * y + a.g_at[i] * E * invb;
                        Yk[o] = y;
                        a.o.lz.L[o] = l;
                        if (a.o.lz.W) a.o.lz.W[o] += a.o.lz.coef[(size_t)a.o.k * a.ld + r] * y;
                        if (cp < (int)blockDim.x) part += y * l;
                        else pcarry[cp - blockDim.x] += y * l;   // thread cp - blockDim.x owns this slot
                    }
                }
            }
        }
    }
    __syncthreads();
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

mbd_status launch_exclusive_scan(const int *in, int *out, int n, DevBuf &bsum, cudaStream_t st) {
    const int nb = (n + 4095) / 4096;
    MBD_TRY(bsum.ensure(sizeof(int) * (size_t)std::max(1, nb)));
    if (n > 0) {
        k_scan_block<<<nb, 1024, 0, st>>>(in, out, bsum.as<int>(), n);
        MBD_LAUNCH_CHECK();
    }
    k_scan_sums<<<1, 32, 0, st>>>(bsum.as<int>(), nb, out + n);
    MBD_LAUNCH_CHECK();
    if (n > 0) {
        k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, bsum.as<int>(), n);
        MBD_LAUNCH_CHECK();
    }
    return MBD_OK;
}

template <class T> mbd_status build_pencil_records(mbd_system *s);

template <class T> mbd_status build_spread_matrix(mbd_system *s) {
    PrecData<T> &P = prec<T>(s);
    const Geom g = geom_of(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    if (npts >= 0x7fffffffULL) return MBD_ERR_UNSUPPORTED;
    // every atom's stencil covers p^3 distinct points (K >= 2p), so the matrix
    // has exactly p^3 N records
    const size_t nnz = (size_t)s->p * s->p * s->p * (size_t)s->N;
    if (nnz >= 0x7fffffffULL) return MBD_ERR_UNSUPPORTED;
    MBD_TRY(P.srow.ensure(sizeof(int) * (npts + 1)));
    MBD_TRY(P.srec.ensure(sizeof(SpreadRec<T>) * std::max<size_t>(1, nnz)));
    DevBuf &cnt = s->scan_cnt, &bsum = s->scan_bsum;
    MBD_TRY(cnt.ensure(sizeof(int) * npts));
    const int threads = 256;
    const BinView &B = s->bins;
    const int npb = B.bs1 * B.bs2 * B.bs3;
    if (B.nc1 * B.nc2 * B.nc3 <= kRowsMaxBins && npb <= 1024) {
        // a block per brick
        const unsigned nbricks = (unsigned)(B.nb1 * B.nb2 * B.nb3);
        const unsigned bt = (unsigned)((npb + 31) / 32 * 32);
        k_spread_rows_brick<T, false><<<nbricks, bt, 0, s->stream>>>(g, B, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                                    s->dw64_d.as<double>(), cnt.as<int>(), nullptr);
        MBD_LAUNCH_CHECK();
        MBD_TRY(launch_exclusive_scan(cnt.as<int>(), P.srow.template as<int>(), (int)npts, bsum, s->stream));
        k_spread_rows_brick<T, true><<<nbricks, bt, 0, s->stream>>>(g, B, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                                   s->dw64_d.as<double>(), P.srow.template as<int>(),
                                                                   P.srec.template as<SpreadRec<T>>());
        MBD_LAUNCH_CHECK();
        return s->p == kPencilOrder ? build_pencil_records<T>(s) : MBD_OK;
    }
    const unsigned blocks = (unsigned)((npts + threads - 1) / threads);
    k_spread_rows<T, false><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                              s->dw64_d.as<double>(), cnt.as<int>(), nullptr);
    MBD_LAUNCH_CHECK();
    MBD_TRY(launch_exclusive_scan(cnt.as<int>(), P.srow.template as<int>(), (int)npts, bsum, s->stream));
    k_spread_rows<T, true><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                             s->dw64_d.as<double>(), P.srow.template as<int>(),
                                                             P.srec.template as<SpreadRec<T>>());
    MBD_LAUNCH_CHECK();
    return s->p == kPencilOrder ? build_pencil_records<T>(s) : MBD_OK;
}

// The pencil records of spline order 6 (the order of the fused pencil
// spreading): counts, CSR starts, records, and the per-atom k3 stencils.
template <class T> mbd_status build_pencil_records(mbd_system *s) {
    PrecData<T> &P = prec<T>(s);
    const Geom g = geom_of(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    const size_t nnz = (size_t)s->p * s->p * (size_t)s->N;   // each atom covers p^2 pencils (K >= 2p)
    if (npts >= 0x7fffffffULL || nnz >= 0x7fffffffULL) return MBD_ERR_UNSUPPORTED;
    MBD_TRY(P.prow.ensure(sizeof(int) * (npts + 1)));
    MBD_TRY(P.prec.ensure(sizeof(PencilRec<T>) * std::max<size_t>(1, nnz)));
    MBD_TRY(P.k3w.ensure(sizeof(T) * 16 * std::max(1, s->N)));
    DevBuf &cnt = s->scan_cnt, &bsum = s->scan_bsum;
    MBD_TRY(cnt.ensure(sizeof(int) * npts));
    const int threads = 256;
    const unsigned blocks = (unsigned)((npts + threads - 1) / threads);
    k_pencil_rows<T, false><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                              s->dw64_d.as<double>(), cnt.as<int>(), nullptr);
    MBD_LAUNCH_CHECK();
    MBD_TRY(launch_exclusive_scan(cnt.as<int>(), P.prow.template as<int>(), (int)npts, bsum, s->stream));
    k_pencil_rows<T, true><<<blocks, threads, 0, s->stream>>>(g, s->bins, s->top_d.as<int>(), s->w64_d.as<double>(),
                                                             s->dw64_d.as<double>(), P.prow.template as<int>(),
                                                             P.prec.template as<PencilRec<T>>());
    MBD_LAUNCH_CHECK();
    if (s->N > 0) {
        k_pencil_k3w<T><<<(16 * s->N + threads - 1) / threads, threads, 0, s->stream>>>(
            s->N, s->p, s->w64_d.as<double>(), s->dw64_d.as<double>(), P.k3w.template as<T>());
        MBD_LAUNCH_CHECK();
    }
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

// Meshes of at most this many bytes (three quarters of the 129 MB L2) launch
// their FFT passes with programmatic dependence; larger ones plainly.
constexpr size_t kEarlyFFTMaxBytes = 96u << 20;

// FP32 passes and fused spreading over meshes longer than this use tiles of
// 16 complex columns instead of 32: half the shared memory per block, twice
// the resident blocks, which the long (latency-bound) spreading phase needs.
constexpr int kWideTileMaxK = 96;

// Tile width of the fused spreading + k3 pass for V complex probe-pair
// columns: whole tiles only (float 32 or 16, double 16), 0 when none fits.
int sf3_width(const mbd_system *s, int V, int real_bytes) {
    if (real_bytes == 4) {
        if (s->tune_sf3_w != 0 && s->tune_ld == 2 * V && V % s->tune_sf3_w == 0) return s->tune_sf3_w;
        return (V % 32 == 0 && s->K[2] <= kWideTileMaxK) ? 32 : (V % 16 == 0 ? 16 : 0);
    }
    return V % 16 == 0 ? 16 : 0;
}

#define MBD_HAS_CASE(K, ...) case K:
bool fft_ct_size(int K) {
    switch (K) {
        MBD_FFT_GROUP0(MBD_HAS_CASE)
        MBD_FFT_GROUP1(MBD_HAS_CASE)
        MBD_FFT_GROUP2(MBD_HAS_CASE)
        MBD_FFT_GROUP3(MBD_HAS_CASE)
        MBD_FFT_GROUP4(MBD_HAS_CASE)
        MBD_FFT_GROUP5(MBD_HAS_CASE)
        return true;
        default: return false;
    }
}
#undef MBD_HAS_CASE

template <class T> int launch_fft_ct_sized(const FFTArgs<T> &a, bool fused, unsigned grid, cudaStream_t st) {
    int r;
    if ((r = launch_fft_ct_group0<T>(a, fused, grid, st)) >= 0) return r;
    if ((r = launch_fft_ct_group1<T>(a, fused, grid, st)) >= 0) return r;
    if ((r = launch_fft_ct_group2<T>(a, fused, grid, st)) >= 0) return r;
    if ((r = launch_fft_ct_group3<T>(a, fused, grid, st)) >= 0) return r;
    if ((r = launch_fft_ct_group4<T>(a, fused, grid, st)) >= 0) return r;
    return launch_fft_ct_group5<T>(a, fused, grid, st);
}

template <class T>
int launch_sf3_sized(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *row,
                     const SpreadRec<T> *rec, const typename Cplx<T>::type *tw, cudaStream_t st) {
    int r;
    if ((r = launch_sf3_group0<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st)) >= 0) return r;
    if ((r = launch_sf3_group1<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st)) >= 0) return r;
    if ((r = launch_sf3_group2<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st)) >= 0) return r;
    if ((r = launch_sf3_group3<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st)) >= 0) return r;
    if ((r = launch_sf3_group4<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st)) >= 0) return r;
    return launch_sf3_group5<T>(K3, W, d, mesh, R, ld, K1, K2, row, rec, tw, st);
}

template <class T>
int launch_spp_sized(int K3, int W, const T *d, T *mesh, int R, int ld, int K1, int K2, const int *prow,
                     const PencilRec<T> *prec, const T *k3w, const typename Cplx<T>::type *tw, cudaStream_t st) {
    int r;
    if ((r = launch_spp_group0<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st)) >= 0) return r;
    if ((r = launch_spp_group1<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st)) >= 0) return r;
    if ((r = launch_spp_group2<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st)) >= 0) return r;
    if ((r = launch_spp_group3<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st)) >= 0) return r;
    if ((r = launch_spp_group4<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st)) >= 0) return r;
    return launch_spp_group5<T>(K3, W, d, mesh, R, ld, K1, K2, prow, prec, k3w, tw, st);
}

// Spreading fused with the first forward FFT pass when the k3 size has a
// compile-time pass and the probe-pair columns fill whole tiles.
bool spread_fft3_supported(const mbd_system *s, int ld, int real_bytes) {
    return fft_ct_size(s->K[2]) && sf3_width(s, ld / 2, real_bytes) > 0;
}

// Returns MBD_ERR_UNSUPPORTED (nothing launched) when spread_fft3_supported is false.
template <class T> mbd_status launch_spread_fft3(mbd_system *s, const T *d, T *mesh, int R, int ld) {
    PrecData<T> &P = prec<T>(s);
    const int W = sf3_width(s, ld / 2, (int)sizeof(T));
    if (W == 0) return MBD_ERR_UNSUPPORTED;
    using C = typename Cplx<T>::type;
    // spline order 6: spreading by pencil records; other orders by the point records
    const int r = s->p == kPencilOrder
                      ? launch_spp_sized<T>(s->K[2], W, d, mesh, R, ld, s->K[0], s->K[1], P.prow.template as<int>(),
                                            P.prec.template as<PencilRec<T>>(), P.k3w.template as<T>(),
                                            P.tw3.template as<C>(), s->stream)
                      : launch_sf3_sized<T>(s->K[2], W, d, mesh, R, ld, s->K[0], s->K[1], P.srow.template as<int>(),
                                            P.srec.template as<SpreadRec<T>>(), P.tw3.template as<C>(), s->stream);
    if (r < 0) return MBD_ERR_UNSUPPORTED;
    if (r == 0) {
        set_last_error("fused spreading: shared-memory size", cudaGetLastError());
        return MBD_ERR_CUDA;
    }
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

template <class T> mbd_status launch_convolve(mbd_system *s, T *mesh, int ld, bool skip_first) {
    using C = typename Cplx<T>::type;
    PrecData<T> &P = prec<T>(s);
    const int V = ld / 2;
    const int K1 = s->K[0], K2 = s->K[1], K3 = s->K[2];
    const int Wmax = sizeof(T) == 4 ? 32 : 16;
    const size_t npts_bytes = sizeof(T) * (size_t)K1 * K2 * K3 * ld;
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
        // early launch of the passes while the mesh fits in three quarters of L2
        a.early = npts_bytes <= kEarlyFFTMaxBytes ? 1 : 0;
        a.sms = s->num_sms;
        // compile-time pass: float tiles of 32 complex columns (16 for narrow
        // rows and for long meshes), double tiles of 16; narrower rows are masked
        FFTArgs<T> c = a;
        c.W = (sizeof(T) == 4 && (inner < 32 || a.K > kWideTileMaxK)) ? 16 : Wmax;
        if (sizeof(T) == 4 && s->tune_fft_w != 0 && s->tune_ld == ld) c.W = inner < 32 ? 16 : s->tune_fft_w;
        // the pass fused with G does twice the arithmetic per element of the
        // mesh: on meshes of 97 to 128 points it keeps 32-column tiles (128^3,
        // 128 probes: 474 -> 462 us per pass on average over the four passes);
        // longer ones do not (192^3: 818 -> 934 us, the tile's shared memory
        // leaves too few blocks per SM)
        if (sizeof(T) == 4 && fused && a.K > kWideTileMaxK && a.K <= 128 && inner >= 32) c.W = 32;
        const int r = launch_fft_ct_sized<T>(c, fused, (unsigned)((size_t)outer * ((inner + c.W - 1) / c.W)),
                                             s->stream);
        if (r == 0) {
            set_last_error("FFT pass: shared-memory size", cudaGetLastError());
            return MBD_ERR_CUDA;
        }
        if (r == 1) {
            MBD_LAUNCH_CHECK();
            return MBD_OK;
        }
        const size_t smem = sizeof(C) * (2 * (size_t)a.K * a.W + a.K);
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
    a.ereal = real_on_clusters(s, ld, (int)sizeof(T)) ? P.ereal.template as<T>() : nullptr;
    a.o = o;
    const int vec = field_vec(ld, (int)sizeof(T));
    const int apb = field_apb(s, ld);
    dim3 grid(field_blocks(s, ld), (ld + 32 * vec - 1) / (32 * vec));
    const bool six = a.ereal != nullptr && s->p == 6;
#define MBD_FIELD_LAUNCH(V, P, NW) k_field<T, V, P, NW><<<grid, (NW) * 32, 0, s->stream>>>(a, apb)
    if constexpr (sizeof(T) == 4) {
        if (six && field_half(ld, 4)) {
            // 64-probe chunks as with two probes per lane, here four probes per
            // lane on half-warps, one atom each
            k_field<T, 4, 6, 6, 16><<<grid, 6 * 32, 0, s->stream>>>(a, apb);
            MBD_LAUNCH_CHECK();
            return MBD_OK;
        }
    }
    if (vec == 4) {
        if constexpr (sizeof(T) == 4) {
            if (six) MBD_FIELD_LAUNCH(4, 6, 6);
            else if (s->p == 6) MBD_FIELD_LAUNCH(4, 6, kWarps);
            else MBD_FIELD_LAUNCH(4, 0, kWarps);
        }
    } else if (vec == 2) {
        if (six) MBD_FIELD_LAUNCH(2, 6, 6);
        else if (s->p == 6) MBD_FIELD_LAUNCH(2, 6, kWarps);
        else MBD_FIELD_LAUNCH(2, 0, kWarps);
    } else {
        if (six) MBD_FIELD_LAUNCH(1, 6, 6);
        else if (s->p == 6) MBD_FIELD_LAUNCH(1, 6, kWarps);
        else MBD_FIELD_LAUNCH(1, 0, kWarps);
    }
#undef MBD_FIELD_LAUNCH
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

// The real-space field runs on the clusters when they were built and there
// are enough of them for four blocks per SM (a block per cluster and probe
// chunk); smaller systems keep the pair loop of the field kernel, whose warps
// split the neighbours of one atom.
bool real_on_clusters(const mbd_system *s, int ld, int real_bytes) {
    if (!s->real_clusters || s->real_method == MBD_REAL_PAIRS) return false;
    if (s->real_method == MBD_REAL_CLUSTERS) return true;
    const int ppl = real_bytes == 4 ? 2 : 1;
    const long long chunks = (ld + 32 * ppl - 1) / (32 * ppl);
    return (long long)s->n_clusters * chunks >= 4LL * std::max(1, s->num_sms);
}

// E_real of every atom from the clusters (the caller runs this before
// launch_field whenever real_on_clusters holds and the real-space term is wanted).
template <class T> mbd_status launch_real_clusters(mbd_system *s, const T *d, T *ereal, int ld, cudaStream_t st) {
    PrecData<T> &P = prec<T>(s);
    RealArgs<T> a;
    a.d = d;
    a.out = ereal;
    a.ld = ld;
    a.N = s->N;
    a.nclus = s->n_clusters;
    a.order = s->order_d.as<int>();
    a.estart = s->cl_estart.as<int>();
    a.pstart = s->cl_pstart.as<int>();
    a.entries = s->cl_entries.as<int>();
    a.pairs = P.cA.template as<RealPair<T>>();
    if (a.nclus == 0) return MBD_OK;
    constexpr int ppl = sizeof(T) == 4 ? 2 : 1;
    dim3 grid((unsigned)a.nclus, (unsigned)((ld + 32 * ppl - 1) / (32 * ppl)));
    const size_t smem = sizeof(T) * kRealCE * 3 * 32 * ppl + sizeof(RealPair<T>) * kClusterSize * 32;
    static bool attr = false;
    if (!attr) {
        MBD_CUDA_TRY(cudaFuncSetAttribute(k_real_clusters<T, ppl>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        attr = true;
    }
    k_real_clusters<T, ppl><<<grid, 32 * kClusterSize, smem, st>>>(a);
    MBD_LAUNCH_CHECK();
    return MBD_OK;
}

// Probes per lane of the field kernel.
int field_vec(int ld, int real_bytes) {
    return (real_bytes == 4 && ld % 4 == 0 && ld >= 128) ? 4 : ((ld % 2 == 0 && ld >= 64) ? 2 : 1);
}

// FP32 chunks of 64 probes (two per lane) whose probe count allows 16-byte
// loads: the six-warp field kernel then gathers one atom per half-warp, four
// probes per lane (the same chunks).
bool field_half(int ld, int real_bytes) { return real_bytes == 4 && field_vec(ld, 4) == 2 && ld % 4 == 0; }

namespace {
// Resident blocks per SM of one field-kernel variant (the same on every
// device of one architecture), asked of the occupancy calculator once.
template <class T, int V, int P, int NW = kWarps, int LPA = 32> int field_occupancy() {
    static int nb = 0;
    if (nb == 0) {
        int x = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x, k_field<T, V, P, NW, LPA>, NW * 32, 0) != cudaSuccess ||
            x < 1) {
            cudaGetLastError();
            x = 1;
        }
        nb = x;
    }
    return nb;
}

int field_resident_blocks(const mbd_system *s, int ld) {
    const bool p6 = s->p == 6;
    const bool fp64 = s->precision == MBD_FP64;
    const bool six = p6 && real_on_clusters(s, ld, fp64 ? 8 : 4);
    int nb;
    if (fp64) {
        const int vec = field_vec(ld, 8);
        if (six)
            nb = vec == 2 ? field_occupancy<double, 2, 6, 6>() : field_occupancy<double, 1, 6, 6>();
        else
            nb = vec == 2 ? (p6 ? field_occupancy<double, 2, 6>() : field_occupancy<double, 2, 0>())
                          : (p6 ? field_occupancy<double, 1, 6>() : field_occupancy<double, 1, 0>());
    } else {
        const int vec = field_vec(ld, 4);
        if (six)
            nb = vec == 4            ? field_occupancy<float, 4, 6, 6>()
                 : field_half(ld, 4) ? field_occupancy<float, 4, 6, 6, 16>()
                 : vec == 2          ? field_occupancy<float, 2, 6, 6>()
                                     : field_occupancy<float, 1, 6, 6>();
        else
            nb = vec == 4   ? (p6 ? field_occupancy<float, 4, 6>() : field_occupancy<float, 4, 0>())
                 : vec == 2 ? (p6 ? field_occupancy<float, 2, 6>() : field_occupancy<float, 2, 0>())
                            : (p6 ? field_occupancy<float, 1, 6>() : field_occupancy<float, 1, 0>());
    }
    return nb * std::max(1, s->num_sms);
}
}  // namespace

// Atoms per block of the field kernel: the blocks fill whole waves of the
// resident-block capacity (blocks per SM x SMs, shared by the probe chunks),
// with at most 64 atoms per block (more waves beyond that, for balance).
int field_apb(const mbd_system *s, int ld) {
    const int bytes = s->precision == MBD_FP64 ? 8 : 4;
    const int vec = field_vec(ld, bytes);
    // the six-warp FP32 kernels take two atoms per iteration: an even count
    // leaves no half-empty iteration
    const bool pairs = bytes == 4 && s->p == 6 && real_on_clusters(s, ld, bytes) && (vec == 4 || field_half(ld, bytes));
    int apb;
    if (s->tune_field_apb > 0 && s->tune_ld == ld) {
        apb = s->tune_field_apb;
    } else {
        const int ych = (ld + 32 * vec - 1) / (32 * vec);
        const long long per_wave = std::max(1, field_resident_blocks(s, ld) / ych);
        const long long waves = (s->N + 64 * per_wave - 1) / (64 * per_wave);
        apb = (int)std::max<long long>(1, (s->N + waves * per_wave - 1) / (waves * per_wave));
    }
    return pairs ? apb + (apb & 1) : apb;
}
int field_blocks(const mbd_system *s, int ld) {
    const int apb = field_apb(s, ld);
    return (s->N + apb - 1) / apb;
}

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
template mbd_status launch_real_clusters<double>(mbd_system *, const double *, double *, int, cudaStream_t);
template mbd_status launch_real_clusters<float>(mbd_system *, const float *, float *, int, cudaStream_t);

}  // namespace mbd
