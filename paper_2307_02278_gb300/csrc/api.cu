// C ABI of libmbd: validation, the per-system setup (neighbour list, spread
// bins, B-spline moduli, FFT plans) and the orchestration of the per-step
// kernels for every entry point declared in include/mbd.h.
#include "mbd_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace mbd {

thread_local std::string g_last_error;

void set_last_error(const char *where, cudaError_t e) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
}

// Host-side failure injection (mbd_debug_fail_allocation): when >= 0, the
// number of device allocations still to succeed before one is reported as
// failed; -1 when disarmed.
std::atomic<long long> g_alloc_countdown{-1};

mbd_status DevBuf::ensure(size_t n) {
    if (ptr != nullptr && n <= bytes) return MBD_OK;
    release();
    if (n == 0) n = 16;
    if (g_alloc_countdown.load() >= 0 && g_alloc_countdown.fetch_sub(1) == 0) {
        g_last_error = "cudaMalloc: allocation failure injected by mbd_debug_fail_allocation";
        return MBD_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(&ptr, n);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        set_last_error("cudaMalloc", e);
        cudaGetLastError();
        return MBD_ERR_OOM;
    }
    bytes = n;
    return MBD_OK;
}

void DevBuf::release() {
    if (ptr != nullptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

void prof_begin(mbd_system *s, int stage, cudaEvent_t *e0) {
    (void)stage;
    *e0 = nullptr;
    if (!s->prof.timing) return;
    Profiler &P = s->prof;
    if (P.pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        P.pool.push_back(e);
    }
    *e0 = P.pool.back();
    P.pool.pop_back();
    cudaEventRecord(*e0, s->stream);
}

void prof_end(mbd_system *s, int stage, int n_launches, cudaEvent_t e0) {
    Profiler &P = s->prof;
    P.launches[stage] += n_launches;
    if (!P.timing || e0 == nullptr) return;
    cudaEvent_t e1;
    if (P.pool.empty()) {
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaGetLastError();
            P.pool.push_back(e0);
            return;
        }
    } else {
        e1 = P.pool.back();
        P.pool.pop_back();
    }
    cudaEventRecord(e1, s->stream);
    P.pending.push_back(Profiler::Rec{stage, e0, e1});
}

// Fold finished event pairs into the per-stage times (after a stream sync).
void prof_collect(mbd_system *s) {
    Profiler &P = s->prof;
    for (const Profiler::Rec &r : P.pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) P.ms[r.stage] += ms;
        cudaGetLastError();
        P.pool.push_back(r.e0);
        P.pool.push_back(r.e1);
    }
    P.pending.clear();
}

void prof_release(mbd_system *s) {
    Profiler &P = s->prof;
    for (const Profiler::Rec &r : P.pending) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    for (cudaEvent_t e : P.pool) cudaEventDestroy(e);
    P.pending.clear();
    P.pool.clear();
}

// gscale kernels live in kernels_lanczos.cu
template <class T> mbd_status launch_gscale(const double *x, const double *g, T *d, int rows, int ld, cudaStream_t st);

namespace {

constexpr double kPi = 3.14159265358979323846;

template <class T> PrecData<T> &prec(mbd_system *s);
template <> PrecData<double> &prec<double>(mbd_system *s) { return s->f64; }
template <> PrecData<float> &prec<float>(mbd_system *s) { return s->f32; }

bool finite_all(const double *x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

// Radices 8, 4, 2, 3, 5 (in that order of preference); false if K has another factor.
bool factor_mesh(int K, FFTDim &f) {
    f.K = K;
    f.nst = 0;
    int k = K;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int r : order) {
        while (k % r == 0) {
            if (f.nst >= kMaxRadixStages) return false;
            f.radix[f.nst++] = r;
            k /= r;
        }
    }
    for (int i = f.nst; i < kMaxRadixStages; ++i) f.radix[i] = 1;
    return k == 1;
}

mbd_status validate(const mbd_system_desc *d) {
    if (d == nullptr) return MBD_ERR_INVALID_ARG;
    if (d->n_atoms < 1 || d->n_atoms > (1 << 24)) return MBD_ERR_INVALID_ARG;
    if (!d->pos || !d->alpha || !d->omega || !d->r_vdw) return MBD_ERR_INVALID_ARG;
    if (!finite_all(d->cell, 9)) return MBD_ERR_INVALID_ARG;
    const double *c = d->cell;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    if (!(det > 0.0)) return MBD_ERR_INVALID_ARG;
    const size_t n = (size_t)d->n_atoms;
    if (!finite_all(d->pos, 3 * n)) return MBD_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; ++i) {
        if (!(d->alpha[i] > 0.0) || !(d->omega[i] > 0.0) || !(d->r_vdw[i] > 0.0)) return MBD_ERR_INVALID_ARG;
        if (!std::isfinite(d->alpha[i]) || !std::isfinite(d->omega[i]) || !std::isfinite(d->r_vdw[i]))
            return MBD_ERR_INVALID_ARG;
    }
    if (!(d->damp_beta > 0.0) || !(d->damp_d > 0.0) || !(d->ewald_beta > 0.0) || !(d->r_cut > 0.0))
        return MBD_ERR_INVALID_ARG;
    if (!std::isfinite(d->damp_beta) || !std::isfinite(d->damp_d) || !std::isfinite(d->ewald_beta) ||
        !std::isfinite(d->r_cut) || !std::isfinite(d->damp_cut))
        return MBD_ERR_INVALID_ARG;
    const int p = d->spline_order;
    if (p < 4 || p > kMaxOrder || (p & 1)) return MBD_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        FFTDim f;
        if (d->mesh[a] < 2 * p || d->mesh[a] > 1000 || !factor_mesh(d->mesh[a], f)) return MBD_ERR_INVALID_ARG;
    }
    if (d->precision != MBD_FP64 && d->precision != MBD_MIXED) return MBD_ERR_INVALID_ARG;
    if (d->quadrature != MBD_QUAD_CHEBYSHEV && d->quadrature != MBD_QUAD_QL && d->quadrature != MBD_QUAD_QL_DF64)
        return MBD_ERR_INVALID_ARG;
    return MBD_OK;
}

void wrap_positions(mbd_system *s, const double *pos) {
    s->pos.resize(3 * (size_t)s->N);
    for (int i = 0; i < s->N; ++i) {
        double f[3];
        for (int a = 0; a < 3; ++a) {
            f[a] = s->recip[3 * a] * pos[3 * i] + s->recip[3 * a + 1] * pos[3 * i + 1] +
                   s->recip[3 * a + 2] * pos[3 * i + 2];
            f[a] -= std::floor(f[a]);
            if (f[a] >= 1.0) f[a] -= 1.0;
        }
        for (int c = 0; c < 3; ++c)
            s->pos[3 * i + c] = f[0] * s->cell[c] + f[1] * s->cell[3 + c] + f[2] * s->cell[6 + c];
    }
}

// Full neighbour list over image pairs (i, j, n) with 0 < |R_i - R_j - n| < rmax
// from a cell list: bins of perpendicular width >= rmax; bin offsets o map to
// (o mod nbins, floor(o / nbins)) = (bin, image), so each (j, n) is visited once.
// Neighbour-list and pair-tensor capacity for nnz pairs, with a quarter more
// room so that small changes of the list between steps need no reallocation.
mbd_status size_pair_buffers(mbd_system *s, long long nnz) {
    const long long cap = std::max<long long>(1, nnz + nnz / 4 + 32);
    MBD_TRY(s->col_d.ensure(sizeof(int) * (size_t)cap));
    MBD_TRY(s->shift_d.ensure(sizeof(int) * (size_t)cap));
    s->nb_cap = cap;
    return MBD_OK;
}

mbd_status build_neighbors(mbd_system *s) {
    const double rmax = std::max(s->r_cut, s->damp_cut);
    const int N = s->N;
    NeighborGrid ng;
    ng.N = N;
    for (int a = 0; a < 3; ++a) {
        const double rn = std::sqrt(s->recip[3 * a] * s->recip[3 * a] + s->recip[3 * a + 1] * s->recip[3 * a + 1] +
                                    s->recip[3 * a + 2] * s->recip[3 * a + 2]);
        const double width = 1.0 / rn;
        ng.nc[a] = std::max(1, std::min(256, (int)std::floor(width / rmax)));
        ng.kk[a] = (int)std::ceil(rmax * ng.nc[a] / width - 1e-12);
        if (ng.kk[a] > 120) return MBD_ERR_INVALID_ARG;
    }
    // cell binning on the host (O(N)), the pair search on the device
    const int ncell = ng.nc[0] * ng.nc[1] * ng.nc[2];
    std::vector<int> bin(N), cstart(ncell + 1, 0), catoms(N), cidx(3 * (size_t)N);
    for (int i = 0; i < N; ++i) {
        int b[3];
        for (int a = 0; a < 3; ++a) {
            double f = s->recip[3 * a] * s->pos[3 * i] + s->recip[3 * a + 1] * s->pos[3 * i + 1] +
                       s->recip[3 * a + 2] * s->pos[3 * i + 2];
            f -= std::floor(f);
            b[a] = std::min(ng.nc[a] - 1, std::max(0, (int)std::floor(f * ng.nc[a])));
            cidx[3 * i + a] = b[a];
        }
        bin[i] = (b[0] * ng.nc[1] + b[1]) * ng.nc[2] + b[2];
        cstart[bin[i] + 1]++;
    }
    for (int c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int> fill(cstart.begin(), cstart.end() - 1);
        for (int i = 0; i < N; ++i) catoms[fill[bin[i]]++] = i;
    }
    MBD_TRY(s->cell_start_d.ensure(sizeof(int) * (ncell + 1)));
    MBD_TRY(s->cell_atoms_d.ensure(sizeof(int) * std::max(1, N)));
    MBD_TRY(s->cell_idx_d.ensure(sizeof(int) * 3 * std::max<size_t>(1, N)));
    MBD_TRY(s->nb_err_d.ensure(sizeof(int)));
    MBD_TRY(s->row_d.ensure(sizeof(int) * (N + 1)));
    MBD_CUDA_TRY(cudaMemcpyAsync(s->cell_start_d.ptr, cstart.data(), sizeof(int) * (ncell + 1),
                                 cudaMemcpyHostToDevice, s->stream));
    MBD_CUDA_TRY(cudaMemcpyAsync(s->cell_atoms_d.ptr, catoms.data(), sizeof(int) * N, cudaMemcpyHostToDevice,
                                 s->stream));
    MBD_CUDA_TRY(cudaMemcpyAsync(s->cell_idx_d.ptr, cidx.data(), sizeof(int) * 3 * N, cudaMemcpyHostToDevice,
                                 s->stream));
    MBD_CUDA_TRY(cudaMemsetAsync(s->nb_err_d.ptr, 0, sizeof(int), s->stream));
    ng.start = s->cell_start_d.as<int>();
    ng.atoms = s->cell_atoms_d.as<int>();
    ng.cidx = s->cell_idx_d.as<int>();
    for (int k = 0; k < 9; ++k) ng.cell[k] = s->cell[k];
    ng.r2max = rmax * rmax;
    s->ngrid = ng;
    MBD_TRY(s->scan_cnt.ensure(sizeof(int) * std::max(1, N)));
    MBD_TRY(launch_neighbors(ng, s->pos_d.as<double>(), s->scan_cnt.as<int>(), nullptr, nullptr,
                             s->nb_err_d.as<int>(), false, 0, s->stream));
    MBD_TRY(launch_exclusive_scan(s->scan_cnt.as<int>(), s->row_d.as<int>(), N, s->scan_bsum, s->stream));
    if (s->nb_cap == 0) {
        // first build: the list is sized from its count (with room to grow)
        int head[2] = {0, 0};
        MBD_CUDA_TRY(cudaMemcpyAsync(&head[0], s->row_d.as<int>() + N, sizeof(int), cudaMemcpyDeviceToHost,
                                     s->stream));
        MBD_CUDA_TRY(cudaMemcpyAsync(&head[1], s->nb_err_d.ptr, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (head[0] < 0 || head[1] != 0) return MBD_ERR_INVALID_ARG;
        MBD_TRY(size_pair_buffers(s, head[0]));
    }
    // later builds keep the buffers and find out at the end whether the list
    // still fits them (setup_geometry)
    return launch_neighbors(ng, s->pos_d.as<double>(), s->row_d.as<int>(), s->col_d.as<int>(),
                            s->shift_d.as<int>(), s->nb_err_d.as<int>(), true, s->nb_cap, s->stream);
}

// Bricks of the mesh for deterministic spreading; atoms are binned by the
// brick of their last stencil point (top), read back from the device so that
// the host and the kernels agree exactly.
mbd_status build_bins(mbd_system *s) {
    const int N = s->N;
    int bs[3], nb[3], ncand[3];
    for (int a = 0; a < 3; ++a) {
        const int K = s->K[a];
        const int pref[5] = {4, 5, 3, 2, 1};
        bs[a] = 1;
        for (int e : pref)
            if (K % e == 0) {
                bs[a] = e;
                break;
            }
        nb[a] = K / bs[a];
        ncand[a] = std::min(nb[a], 1 + (bs[a] + s->p - 2) / bs[a]);
    }
    const int nbins = nb[0] * nb[1] * nb[2];
    MBD_TRY(s->bin_start_d.ensure(sizeof(int) * (nbins + 1)));
    MBD_TRY(s->bin_atoms_d.ensure(sizeof(int) * std::max(1, N)));
    MBD_TRY(s->order_d.ensure(sizeof(int) * std::max(1, N)));
    MBD_TRY(s->bin_of_d.ensure(sizeof(int) * std::max(1, N)));
    MBD_TRY(s->bin_cursor_d.ensure(sizeof(int) * nbins));
    MBD_TRY(s->scan_cnt.ensure(sizeof(int) * std::max(nbins, N)));
    BinView &B = s->bins;
    B.nb1 = nb[0];
    B.nb2 = nb[1];
    B.nb3 = nb[2];
    B.bs1 = bs[0];
    B.bs2 = bs[1];
    B.bs3 = bs[2];
    B.nc1 = ncand[0];
    B.nc2 = ncand[1];
    B.nc3 = ncand[2];
    B.start = s->bin_start_d.as<int>();
    B.atoms = s->bin_atoms_d.as<int>();
    MBD_TRY(launch_bin_atoms(N, s->top_d.as<int>(), B, s->bin_of_d.as<int>(), s->scan_cnt.as<int>(),
                             s->bin_start_d.as<int>(), s->bin_cursor_d.as<int>(), s->bin_atoms_d.as<int>(),
                             s->scan_bsum, s->stream));
    // the field kernel and the real-space clusters take the atoms in the
    // Morton order of their bricks (compact groups of consecutive atoms); a
    // brick grid too large for the Morton cube keeps the brick-major order
    const mbd_status mo = launch_morton_order(B, N, s->order_d.as<int>(), s->morton_cnt, s->morton_start,
                                              s->scan_bsum, s->stream);
    if (mo == MBD_ERR_UNSUPPORTED && N > 0)
        MBD_CUDA_TRY(cudaMemcpyAsync(s->order_d.ptr, s->bin_atoms_d.ptr, sizeof(int) * N, cudaMemcpyDeviceToDevice,
                                     s->stream));
    else if (mo != MBD_OK)
        return mo;
    return MBD_OK;
}

// M_p at the integers 0..p (recursion from M_2), for the B-spline moduli.
void bspline_integers(int p, double *out) {
    std::vector<double> cur(p + 1, 0.0), nxt(p + 1, 0.0);
    cur[1] = 1.0;   // M_2(0) = 0, M_2(1) = 1, M_2(2) = 0
    for (int n = 3; n <= p; ++n) {
        for (int k = 0; k <= p; ++k) {
            const double a = (k < p + 1) ? cur[k] : 0.0;
            const double b = (k >= 1) ? cur[k - 1] : 0.0;
            nxt[k] = (k * a + (n - k) * b) / (n - 1);
        }
        cur = nxt;
    }
    for (int k = 0; k <= p; ++k) out[k] = cur[k];
}

// |b(m)|^2 = 1 / |sum_{j=0}^{p-2} M_p(j+1) exp(2 pi i m j / K)|^2
void bspline_moduli(int K, int p, double *out) {
    std::vector<double> mi(p + 1);
    bspline_integers(p, mi.data());
    for (int m = 0; m < K; ++m) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j <= p - 2; ++j) {
            const double ang = 2.0 * kPi * (double)((long long)m * j % K) / K;
            re += mi[j + 1] * std::cos(ang);
            im += mi[j + 1] * std::sin(ang);
        }
        out[m] = 1.0 / (re * re + im * im);
    }
}

template <class T> mbd_status upload_twiddles(mbd_system *s) {
    using C = typename Cplx<T>::type;
    PrecData<T> &P = prec<T>(s);
    DevBuf *tw[3] = {&P.tw1, &P.tw2, &P.tw3};
    for (int a = 0; a < 3; ++a) {
        const int K = s->K[a];
        std::vector<C> h(K);
        for (int n = 0; n < K; ++n) {
            const double ang = 2.0 * kPi * n / K;
            h[n].x = T(std::cos(ang));
            h[n].y = T(-std::sin(ang));
        }
        MBD_TRY(tw[a]->ensure(sizeof(C) * K));
        MBD_CUDA_TRY(cudaMemcpyAsync(tw[a]->ptr, h.data(), sizeof(C) * K, cudaMemcpyHostToDevice, s->stream));
        MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    }
    return MBD_OK;
}

// Positions to neighbour list, pair tensors, splines, bricks and spreading
// matrix, all queued on the stream; one readback at the end gives the pair
// count and the error flags.  A list that outgrew its buffers is filled again
// into larger ones, with its pair tensors.
template <class T> mbd_status setup_geometry(mbd_system *s) {
    MBD_CUDA_TRY(cudaMemcpyAsync(s->pos_d.ptr, s->pos.data(), sizeof(double) * 3 * s->N, cudaMemcpyHostToDevice,
                                 s->stream));
    MBD_TRY(build_neighbors(s));
    MBD_TRY(launch_pair_tensors<T>(s, s->stream));
    MBD_TRY(launch_splines<T>(s, s->stream));
    MBD_TRY(build_bins(s));
    MBD_TRY(build_spread_matrix<T>(s));
    int head[2] = {0, 0};
    MBD_CUDA_TRY(cudaMemcpyAsync(&head[0], s->row_d.as<int>() + s->N, sizeof(int), cudaMemcpyDeviceToHost,
                                 s->stream));
    MBD_CUDA_TRY(cudaMemcpyAsync(&head[1], s->nb_err_d.ptr, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (head[0] < 0 || head[1] != 0) return MBD_ERR_INVALID_ARG;
    s->nnz = head[0];
    if (s->nnz > s->nb_cap) {
        MBD_TRY(size_pair_buffers(s, s->nnz));
        MBD_TRY(launch_neighbors(s->ngrid, s->pos_d.as<double>(), s->row_d.as<int>(), s->col_d.as<int>(),
                                 s->shift_d.as<int>(), s->nb_err_d.as<int>(), true, s->nb_cap, s->stream));
        MBD_TRY(launch_pair_tensors<T>(s, s->stream));
    }
    // the clusters of the real-space field, from the final neighbour list
    s->real_clusters = false;
    s->n_clusters = (s->N + kClusterSize - 1) / kClusterSize;
    MBD_TRY(s->cl_err.ensure(sizeof(int)));
    MBD_CUDA_TRY(cudaMemsetAsync(s->cl_err.ptr, 0, sizeof(int), s->stream));
    MBD_TRY(launch_cluster_pairs<T>(s, s->order_d.as<int>(), s->n_clusters, s->cl_ecnt, s->cl_pcnt, s->cl_estart,
                                    s->cl_pstart, s->cl_entries, prec<T>(s).cA, s->cl_err.as<int>(), s->stream));
    int cerr = 0;
    MBD_CUDA_TRY(cudaMemcpyAsync(&cerr, s->cl_err.ptr, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->real_clusters = cerr == 0;
    return MBD_OK;
}

template <class T> mbd_status setup_mesh(mbd_system *s) {
    std::vector<double> bm(s->K[0] + s->K[1] + s->K[2]);
    bspline_moduli(s->K[0], s->p, bm.data());
    bspline_moduli(s->K[1], s->p, bm.data() + s->K[0]);
    bspline_moduli(s->K[2], s->p, bm.data() + s->K[0] + s->K[1]);
    MBD_TRY(launch_influence<T>(s, bm.data(), s->stream));
    MBD_TRY(upload_twiddles<T>(s));
    return MBD_OK;
}

mbd_status create_impl(const mbd_system_desc *d, void *stream, mbd_system **out) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        if (e != cudaSuccess) set_last_error("cudaGetDeviceCount", e);
        cudaGetLastError();
        return MBD_ERR_NO_DEVICE;
    }
    mbd_system *s = new (std::nothrow) mbd_system();
    if (!s) return MBD_ERR_OOM;
    s->N = d->n_atoms;
    std::memcpy(s->cell, d->cell, sizeof(s->cell));
    // reciprocal rows a*_alpha with a*_alpha . a_beta = delta: inverse transpose of the cell
    const double *c = s->cell;
    const double det = c[0] * (c[4] * c[8] - c[5] * c[7]) - c[1] * (c[3] * c[8] - c[5] * c[6]) +
                       c[2] * (c[3] * c[7] - c[4] * c[6]);
    s->volume = det;
    double inv[9];
    inv[0] = (c[4] * c[8] - c[5] * c[7]) / det;
    inv[1] = (c[2] * c[7] - c[1] * c[8]) / det;
    inv[2] = (c[1] * c[5] - c[2] * c[4]) / det;
    inv[3] = (c[5] * c[6] - c[3] * c[8]) / det;
    inv[4] = (c[0] * c[8] - c[2] * c[6]) / det;
    inv[5] = (c[2] * c[3] - c[0] * c[5]) / det;
    inv[6] = (c[3] * c[7] - c[4] * c[6]) / det;
    inv[7] = (c[1] * c[6] - c[0] * c[7]) / det;
    inv[8] = (c[0] * c[4] - c[1] * c[3]) / det;
    // recip row alpha = column alpha of inv (cell^-1)
    for (int a = 0; a < 3; ++a)
        for (int x = 0; x < 3; ++x) s->recip[3 * a + x] = inv[3 * x + a];
    for (int a = 0; a < 3; ++a) {
        s->K[a] = d->mesh[a];
        factor_mesh(s->K[a], s->fft[a]);
    }
    s->p = d->spline_order;
    s->ewald_beta = d->ewald_beta;
    s->r_cut = d->r_cut;
    s->damp_cut = d->damp_cut > 0.0 ? d->damp_cut : d->r_cut;
    s->damp_beta = d->damp_beta;
    s->damp_d = d->damp_d;
    s->precision = d->precision;
    s->quad_method = d->quadrature;
    s->stream = static_cast<cudaStream_t>(stream);
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            s->num_sms = nsm;
        cudaGetLastError();
    }
    const size_t n = (size_t)s->N;
    s->alpha.assign(d->alpha, d->alpha + n);
    s->omega.assign(d->omega, d->omega + n);
    s->rvdw.assign(d->r_vdw, d->r_vdw + n);
    s->omega_sum = 0.0;
    for (size_t i = 0; i < n; ++i) s->omega_sum += s->omega[i];
    wrap_positions(s, d->pos);
    std::vector<double> g(n), w2(n);
    for (size_t i = 0; i < n; ++i) {
        g[i] = s->omega[i] * std::sqrt(s->alpha[i]);
        w2[i] = s->omega[i] * s->omega[i];
    }
    auto fail = [&](mbd_status st) {
        mbd_destroy_system(s);
        return st;
    };
    mbd_status st;
    if ((st = s->pos_d.ensure(sizeof(double) * 3 * n)) != MBD_OK) return fail(st);
    if ((st = s->g_d.ensure(sizeof(double) * n)) != MBD_OK) return fail(st);
    if ((st = s->w2_d.ensure(sizeof(double) * n)) != MBD_OK) return fail(st);
    if ((st = s->rvdw_d.ensure(sizeof(double) * n)) != MBD_OK) return fail(st);
    if ((st = s->top_d.ensure(sizeof(int) * 3 * n)) != MBD_OK) return fail(st);
    if (cudaMallocHost(&s->host_scal, 16 * sizeof(double)) != cudaSuccess) {
        s->host_scal = nullptr;
        cudaGetLastError();
        return fail(MBD_ERR_OOM);
    }
    if (cudaMallocHost(&s->host_status, 4 * sizeof(int)) != cudaSuccess) {
        s->host_status = nullptr;
        cudaGetLastError();
        return fail(MBD_ERR_OOM);
    }
    cudaError_t ce;
    if ((ce = cudaMemcpyAsync(s->g_d.ptr, g.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->stream)) ||
        (ce = cudaMemcpyAsync(s->w2_d.ptr, w2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->stream)) ||
        (ce = cudaMemcpyAsync(s->rvdw_d.ptr, s->rvdw.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                              s->stream)) ||
        (ce = cudaStreamSynchronize(s->stream))) {
        set_last_error("upload", ce);
        return fail(MBD_ERR_CUDA);
    }
    if (s->precision == MBD_FP64) {
        if ((st = setup_geometry<double>(s)) != MBD_OK) return fail(st);
        if ((st = setup_mesh<double>(s)) != MBD_OK) return fail(st);
    } else {
        if ((st = setup_geometry<float>(s)) != MBD_OK) return fail(st);
        if ((st = setup_mesh<float>(s)) != MBD_OK) return fail(st);
    }
    *out = s;
    return MBD_OK;
}

// ---------------------------------------------------------------- Lanczos workspace
struct Lz {
    LanczosView v;
    int R, ld, m, rows, nblk;
};

mbd_status lanczos_workspace(mbd_system *s, int R, int m, int rows, int field_nblk, Lz &z) {
    z.R = R;
    z.ld = probe_ld(R);
    z.m = m;
    z.rows = rows;
    // prologue blocks per probe chunk: one per SM (fewer, fuller blocks keep the
    // two-level norm reduction short), at least 16 rows each; vectors of more
    // than 2^22 values take two to four per SM, so that enough loads are in
    // flight to stream them from HBM
    const long long vals = (long long)rows * probe_ld(R);
    const int per_sm = vals >= (1LL << 24) ? 4 : (vals >= (1LL << 22) ? 2 : 1);
    z.nblk = std::max(1, std::min((rows + 15) / 16, per_sm * std::max(1, s->num_sms)));
    const size_t ld = z.ld;
    const int nchunk = (z.ld + 31) / 32;
    const int slots = s->basis_recompute ? std::min(3, m) : m;
    MBD_TRY(s->Y.ensure(sizeof(double) * (size_t)slots * rows * ld));
    MBD_TRY(s->L.ensure(sizeof(double) * (size_t)rows * ld));
    MBD_TRY(s->a.ensure(sizeof(double) * (size_t)m * ld));
    MBD_TRY(s->b.ensure(sizeof(double) * (size_t)m * ld));
    MBD_TRY(s->invb.ensure(sizeof(double) * ld));
    MBD_TRY(s->length.ensure(sizeof(int) * ld));
    const int maxblk = std::max(z.nblk, field_nblk);
    const int ngroups = (maxblk + kRedGroup - 1) / kRedGroup;
    MBD_TRY(s->partial.ensure(sizeof(double) * (size_t)maxblk * ld));
    MBD_TRY(s->gpartial.ensure(sizeof(double) * (size_t)ngroups * ld));
    z.v.cstride = ngroups + 1;
    // probe chunks of 32 (prologue) or 32 * VEC (field): 32 is the finest
    const size_t cbytes = sizeof(unsigned) * (size_t)nchunk * z.v.cstride;
    if (s->counter.bytes < cbytes || s->counter_stride != z.v.cstride) {
        MBD_TRY(s->counter.ensure(cbytes));
        MBD_CUDA_TRY(cudaMemsetAsync(s->counter.ptr, 0, s->counter.bytes, s->stream));
        s->counter_stride = z.v.cstride;
    }
    MBD_TRY(s->q.ensure(sizeof(double) * ld));
    MBD_TRY(s->scal.ensure(sizeof(double) * 16));
    MBD_TRY(s->status.ensure(sizeof(int) * 4));
    MBD_TRY(s->qflag.ensure(sizeof(int) * ld));
    z.v.Y = s->Y.as<double>();
    z.v.L = s->L.as<double>();
    z.v.a = s->a.as<double>();
    z.v.b = s->b.as<double>();
    z.v.invb = s->invb.as<double>();
    z.v.length = s->length.as<int>();
    z.v.partial = s->partial.as<double>();
    z.v.gpartial = s->gpartial.as<double>();
    z.v.counter = s->counter.as<unsigned>();
    z.v.yslots = slots;
    z.v.W = nullptr;
    z.v.coef = nullptr;
    return MBD_OK;
}

template <class T> mbd_status ensure_mesh(mbd_system *s, int ld) {
    PrecData<T> &P = prec<T>(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    MBD_TRY(P.d.ensure(sizeof(T) * 3 * (size_t)s->N * ld));
    MBD_TRY(P.mesh.ensure(sizeof(T) * npts * ld));
    if (s->real_clusters) MBD_TRY(P.ereal.ensure(sizeof(T) * 3 * (size_t)s->N * ld));
    return MBD_OK;
}

// Workspace for an m-step run with R probes (allocations only: eager).
template <class T> mbd_status prepare_lanczos(mbd_system *s, int R, int m, Lz &z, bool full) {
    const int rows = 3 * s->N;
    MBD_TRY(lanczos_workspace(s, R, m, rows, field_blocks(s, probe_ld(R)), z));
    MBD_TRY(ensure_mesh<T>(s, z.ld));
    if (full) MBD_TRY(s->work2.ensure(sizeof(double) * (size_t)m * z.ld));
    return MBD_OK;
}

// The m steps of the recurrence (prologue, spreading, FFT convolution, field
// kernel).  v0 (device [3N][ld], may be null) receives y_0 after the first step.
template <class T>
mbd_status enqueue_steps(mbd_system *s, int R, int m, uint64_t seed, const uint64_t *seed_dev, const Lz &z,
                         double *v0) {
    const int rows = 3 * s->N;
    PrecData<T> &P = prec<T>(s);
    FieldOut<T> fo;
    fo.mode = kFieldLanczos;
    fo.terms = MBD_TERM_ALL;
    fo.out = nullptr;
    fo.xin = nullptr;
    fo.lz = z.v;
    // the fused spread + k3 pass exists for the specialised sizes with whole probe-pair tiles
    const bool fuse3 = spread_fft3_supported(s, z.ld, (int)sizeof(T));
    const bool real_cl = real_on_clusters(s, z.ld, (int)sizeof(T));
    for (int k = 0; k < m; ++k) {
        MBD_STAGE(s, MBD_STAGE_PROLOGUE, 1,
                  launch_prologue_t(s->stream, z.v, k, m, seed, R, z.ld, rows, s->g_d.as<double>(), P.d.ptr,
                                    (int)sizeof(T), z.nblk, seed_dev));
        MBD_STAGE(s, MBD_STAGE_SPREAD, 1,
                  fuse3 ? launch_spread_fft3<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, z.ld)
                        : launch_spread<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, z.ld));
        MBD_STAGE(s, MBD_STAGE_FFT, fuse3 ? 4 : 5, launch_convolve<T>(s, P.mesh.template as<T>(), z.ld, fuse3));
        fo.k = k;
        if (real_cl)
            MBD_STAGE(s, MBD_STAGE_REAL, 1,
                      launch_real_clusters<T>(s, P.d.template as<T>(), P.ereal.template as<T>(), z.ld, s->stream));
        MBD_STAGE(s, MBD_STAGE_FIELD, 1,
                  launch_field<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, z.ld, fo));
        if (k == 0 && v0)
            MBD_CUDA_TRY(cudaMemcpyAsync(v0, z.v.Y, sizeof(double) * (size_t)rows * z.ld, cudaMemcpyDeviceToDevice,
                                         s->stream));
    }
    return MBD_OK;
}

// Algorithm 1 with Algorithm 2 per step: m Lanczos steps for all R probes, the
// quadrature and the energy, enqueued on s->stream (kernels and memsets only,
// so the sequence can be captured in a CUDA graph).  seed_dev, when set, is a
// device word holding the seed (read by the first prologue).
template <class T>
mbd_status enqueue_lanczos(mbd_system *s, int R, int m, uint64_t seed, const uint64_t *seed_dev, const Lz &z,
                           bool full) {
    const int rows = 3 * s->N;
    MBD_CUDA_TRY(cudaMemsetAsync(s->a.ptr, 0, sizeof(double) * (size_t)m * z.ld, s->stream));
    MBD_CUDA_TRY(cudaMemsetAsync(s->b.ptr, 0, sizeof(double) * (size_t)m * z.ld, s->stream));
    MBD_CUDA_TRY(cudaMemsetAsync(s->status.ptr, 0, sizeof(int) * 4, s->stream));
    MBD_TRY(enqueue_steps<T>(s, R, m, seed, seed_dev, z, nullptr));
    MBD_STAGE(s, MBD_STAGE_QUADRATURE, 1,
              launch_quadrature(z.v.a, z.v.b, z.v.length, R, z.ld, m, s->q.as<double>(),
                                full ? s->work2.as<double>() : nullptr, s->status.as<int>(), s->qflag.as<int>(),
                                s->stream, s->quad_method));
    MBD_STAGE(s, MBD_STAGE_QUADRATURE, 1,
              launch_energy_reduce(s->q.as<double>(), R, rows, s->omega_sum, s->scal.as<double>(), s->stream));
    return MBD_OK;
}

template <class T> mbd_status run_lanczos(mbd_system *s, int R, int m, uint64_t seed, Lz &z, bool full = false) {
    MBD_TRY(prepare_lanczos<T>(s, R, m, z, full));
    return enqueue_lanczos<T>(s, R, m, seed, nullptr, z, full);
}

mbd_status status_from_bits(int bits) {
    if (bits & 1) return MBD_ERR_NOT_POSITIVE_DEFINITE;
    if (bits & 6) return MBD_ERR_NONFINITE;
    return MBD_OK;
}

// Copy energy, trace, status, and optionally q and (a, b) to the host.
mbd_status fetch_results(mbd_system *s, const Lz &z, double *energy, double *trace, double *q_host,
                         double *ab_host) {
    MBD_CUDA_TRY(cudaMemcpyAsync(s->host_scal, s->scal.ptr, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    MBD_CUDA_TRY(cudaMemcpyAsync(s->host_status, s->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    std::vector<double> qv, av, bv;
    if (q_host) {
        qv.resize(z.R);
        MBD_CUDA_TRY(cudaMemcpyAsync(qv.data(), s->q.ptr, sizeof(double) * z.R, cudaMemcpyDeviceToHost, s->stream));
    }
    if (ab_host) {
        av.resize((size_t)z.m * z.ld);
        bv.resize((size_t)z.m * z.ld);
        MBD_CUDA_TRY(cudaMemcpyAsync(av.data(), s->a.ptr, sizeof(double) * av.size(), cudaMemcpyDeviceToHost,
                                     s->stream));
        MBD_CUDA_TRY(cudaMemcpyAsync(bv.data(), s->b.ptr, sizeof(double) * bv.size(), cudaMemcpyDeviceToHost,
                                     s->stream));
    }
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    prof_collect(s);
    const mbd_status st = status_from_bits(*s->host_status);
    if (st != MBD_OK) return st;
    if (!std::isfinite(s->host_scal[0])) return MBD_ERR_NONFINITE;
    *energy = s->host_scal[0];
    if (trace) *trace = s->host_scal[1];
    if (q_host) std::memcpy(q_host, qv.data(), sizeof(double) * z.R);
    if (ab_host) {
        for (int r = 0; r < z.R; ++r)
            for (int k = 0; k < z.m; ++k) {
                ab_host[((size_t)r * 2) * z.m + k] = av[(size_t)k * z.ld + r];
                ab_host[((size_t)r * 2 + 1) * z.m + k] = bv[(size_t)k * z.ld + r];
            }
    }
    return MBD_OK;
}

template <class T>
mbd_status energy_impl(mbd_system *s, int R, int m, uint64_t seed, double *energy, double *trace, double *q_host,
                       double *ab_host) {
    Lz z;
    MBD_TRY(run_lanczos<T>(s, R, m, seed, z));
    return fetch_results(s, z, energy, trace, q_host, ab_host);
}

template <class T>
mbd_status forces_impl(mbd_system *s, int R, int m, uint64_t seed, double *energy, double *forces_dev) {
    Lz z;
    // w_l = C^{-1/2} v_l = sum_k c_lk y_lk with c = Delta^{-1/2} e_1 from the quadrature kernel
    MBD_TRY(run_lanczos<T>(s, R, m, seed, z, true));
    PrecData<T> &P = prec<T>(s);
    const int ld2 = 2 * R;
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    MBD_TRY(P.d.ensure(sizeof(T) * 3 * (size_t)s->N * std::max(ld2, z.ld)));
    MBD_TRY(P.mesh.ensure(sizeof(T) * npts * std::max(ld2, z.ld)));
    if (s->basis_recompute) {
        // rerun the recurrence (same kernels in the same order: the same y_k),
        // adding c_k y_k into w as each y_k is completed
        const size_t vbytes = sizeof(double) * 3 * (size_t)s->N * z.ld;
        MBD_TRY(s->wacc.ensure(vbytes));
        MBD_TRY(s->v0.ensure(vbytes));
        MBD_CUDA_TRY(cudaMemsetAsync(s->wacc.ptr, 0, vbytes, s->stream));
        Lz z2 = z;
        z2.v.W = s->wacc.as<double>();
        z2.v.coef = s->work2.as<double>();
        MBD_TRY(enqueue_steps<T>(s, R, m, seed, nullptr, z2, s->v0.as<double>()));
        MBD_STAGE(s, MBD_STAGE_FORCE_PREP, 1,
                  launch_force_dipoles_w_t<T>(s, s->wacc.as<double>(), s->v0.as<double>(), R, z.ld,
                                              P.d.template as<T>(), ld2));
    } else {
        MBD_STAGE(s, MBD_STAGE_FORCE_PREP, 1,
                  launch_force_dipoles_t<T>(s, z.v.Y, s->work2.as<double>(), z.v.length, R, z.ld, m,
                                            P.d.template as<T>(), ld2));
    }
    const bool fuse3 = spread_fft3_supported(s, ld2, (int)sizeof(T));
    if (fuse3) {
        MBD_STAGE(s, MBD_STAGE_FORCE_SPREAD, 1,
                  launch_spread_fft3<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), ld2, ld2));
        MBD_STAGE(s, MBD_STAGE_FORCE_FFT, 4, launch_convolve<T>(s, P.mesh.template as<T>(), ld2, true));
    } else {
        MBD_STAGE(s, MBD_STAGE_FORCE_SPREAD, 1,
                  launch_spread<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), ld2, ld2));
        MBD_STAGE(s, MBD_STAGE_FORCE_FFT, 5, launch_convolve<T>(s, P.mesh.template as<T>(), ld2));
    }
    const double scale = 0.25 * (3.0 * s->N) / R;
    MBD_STAGE(s, MBD_STAGE_FORCE_GATHER, 1,
              launch_force_gather_t<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, ld2, scale,
                                       forces_dev));
    return fetch_results(s, z, energy, nullptr, nullptr, nullptr);
}

template <class T> mbd_status apply_impl(mbd_system *s, int nvec, const double *x, double *y, int terms, bool field) {
    const int rows = 3 * s->N;
    const int ld = probe_ld(nvec);
    MBD_TRY(ensure_mesh<T>(s, ld));
    MBD_TRY(s->L.ensure(sizeof(double) * (size_t)rows * ld));
    MBD_TRY(s->work2.ensure(sizeof(double) * (size_t)rows * ld));
    double *xt = s->L.as<double>();
    double *yt = s->work2.as<double>();
    PrecData<T> &P = prec<T>(s);
    MBD_CUDA_TRY(cudaMemsetAsync(xt, 0, sizeof(double) * (size_t)rows * ld, s->stream));
    MBD_STAGE(s, MBD_STAGE_OTHER, 1, launch_to_probe_major(x, nvec, rows, xt, ld, s->stream));
    if (field) {
        MBD_STAGE(s, MBD_STAGE_OTHER, 1, launch_cast_rows<T>(xt, P.d.template as<T>(), (size_t)rows * ld, s->stream));
    } else {
        MBD_STAGE(s, MBD_STAGE_OTHER, 1,
                  launch_gscale<T>(xt, s->g_d.as<double>(), P.d.template as<T>(), rows, ld, s->stream));
    }
    if (terms & MBD_TERM_RECIP) {
        MBD_STAGE(s, MBD_STAGE_SPREAD, 1, launch_spread<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), nvec, ld));
        MBD_STAGE(s, MBD_STAGE_FFT, 5, launch_convolve<T>(s, P.mesh.template as<T>(), ld));
    }
    FieldOut<T> fo;
    fo.mode = field ? kFieldOut : kFieldApply;
    fo.terms = terms;
    fo.out = yt;
    fo.xin = xt;
    fo.k = 0;
    std::memset(&fo.lz, 0, sizeof(fo.lz));
    if (real_on_clusters(s, ld, (int)sizeof(T)) && (terms & MBD_TERM_REAL))
        MBD_STAGE(s, MBD_STAGE_REAL, 1,
                  launch_real_clusters<T>(s, P.d.template as<T>(), P.ereal.template as<T>(), ld, s->stream));
    MBD_STAGE(s, MBD_STAGE_FIELD, 1, launch_field<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), nvec, ld, fo));
    MBD_STAGE(s, MBD_STAGE_OTHER, 1, launch_from_probe_major(yt, nvec, rows, ld, y, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    prof_collect(s);
    return MBD_OK;
}

template <class T> mbd_status spread_impl(mbd_system *s, int nvec, const double *d, double *mesh_out) {
    const int rows = 3 * s->N;
    const int ld = probe_ld(nvec);
    MBD_TRY(ensure_mesh<T>(s, ld));
    MBD_TRY(s->L.ensure(sizeof(double) * (size_t)rows * ld));
    double *xt = s->L.as<double>();
    PrecData<T> &P = prec<T>(s);
    MBD_CUDA_TRY(cudaMemsetAsync(xt, 0, sizeof(double) * (size_t)rows * ld, s->stream));
    MBD_TRY(launch_to_probe_major(d, nvec, rows, xt, ld, s->stream));
    MBD_TRY(launch_cast_rows<T>(xt, P.d.template as<T>(), (size_t)rows * ld, s->stream));
    MBD_TRY(launch_spread<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), nvec, ld));
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    MBD_TRY(launch_mesh_out<T>(P.mesh.template as<T>(), nvec, npts, ld, mesh_out, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return MBD_OK;
}

template <class T> mbd_status convolve_impl(mbd_system *s, int nvec, const double *in, double *out) {
    const int ld = probe_ld(nvec);
    MBD_TRY(ensure_mesh<T>(s, ld));
    PrecData<T> &P = prec<T>(s);
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    MBD_TRY(launch_mesh_in<T>(in, nvec, npts, ld, P.mesh.template as<T>(), s->stream));
    MBD_STAGE(s, MBD_STAGE_FFT, 5, launch_convolve<T>(s, P.mesh.template as<T>(), ld));
    MBD_TRY(launch_mesh_out<T>(P.mesh.template as<T>(), nvec, npts, ld, out, s->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    prof_collect(s);
    return MBD_OK;
}

// ---------------------------------------------------------------- batches of systems
}  // namespace
}  // namespace mbd

struct mbd_batch {
    int n = 0;
    int precision = MBD_FP64;
    long long total_atoms = 0;
    cudaStream_t stream = nullptr;        // caller's stream: graph launches and result copies
    cudaStream_t cap = nullptr;           // capture origin (a capturing stream cannot be the legacy stream)
    std::vector<mbd_system *> sys;
    std::vector<cudaStream_t> streams;    // one per member: its branch of the graph
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    mbd::DevBuf seeds_d, out_d;           // [n] seeds; [n][2] (energy, trace) then [n] status words
    uint64_t *host_seeds = nullptr;
    unsigned char *host_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    int gR = 0, gm = 0;
};

namespace mbd {
namespace {

void destroy_batch_graph(mbd_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_kernels = 0;
    b->gR = b->gm = 0;
}

// Every member's run as one branch: fork from the capture stream, the whole
// Lanczos run on the member's stream, its energy, trace and status copied into
// the batch's output block, join back.
template <class T> mbd_status enqueue_batch(mbd_batch *b, int R, int m, std::vector<Lz> &zs) {
    const size_t n = (size_t)b->n;
    double *out = b->out_d.as<double>();
    int *status = reinterpret_cast<int *>(out + 2 * n);
    MBD_CUDA_TRY(cudaEventRecord(b->fork, b->cap));
    for (size_t i = 0; i < n; ++i) {
        mbd_system *s = b->sys[i];
        MBD_CUDA_TRY(cudaStreamWaitEvent(s->stream, b->fork, 0));
        MBD_TRY(enqueue_lanczos<T>(s, R, m, 0, b->seeds_d.as<uint64_t>() + i, zs[i], false));
        MBD_CUDA_TRY(cudaMemcpyAsync(out + 2 * i, s->scal.ptr, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                     s->stream));
        MBD_CUDA_TRY(cudaMemcpyAsync(status + i, s->status.ptr, sizeof(int), cudaMemcpyDeviceToDevice, s->stream));
        MBD_CUDA_TRY(cudaEventRecord(b->join[i], s->stream));
        MBD_CUDA_TRY(cudaStreamWaitEvent(b->cap, b->join[i], 0));
    }
    return MBD_OK;
}

template <class T> mbd_status capture_batch(mbd_batch *b, int R, int m) {
    destroy_batch_graph(b);
    std::vector<Lz> zs(b->n);
    // allocations (and the counters' one-time clearing) happen eagerly, outside the graph
    for (int i = 0; i < b->n; ++i) {
        MBD_TRY(prepare_lanczos<T>(b->sys[i], R, m, zs[i], false));
        MBD_CUDA_TRY(cudaStreamSynchronize(b->sys[i]->stream));
    }
    MBD_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    const mbd_status st = enqueue_batch<T>(b, R, m, zs);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    if (st != MBD_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (ce != cudaSuccess) set_last_error("cudaStreamEndCapture", ce);
        cudaGetLastError();
        return st != MBD_OK ? st : MBD_ERR_CUDA;
    }
    size_t nnodes = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nnodes);
    std::vector<cudaGraphNode_t> nodes(nnodes);
    if (e == cudaSuccess && nnodes) e = cudaGraphGetNodes(g, nodes.data(), &nnodes);
    long long kernels = 0;
    for (size_t i = 0; e == cudaSuccess && i < nnodes; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        kernels += (t == cudaGraphNodeTypeKernel);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        set_last_error("graph instantiate", e);
        cudaGetLastError();
        return MBD_ERR_CUDA;
    }
    b->graph_kernels = kernels;
    b->gR = R;
    b->gm = m;
    return MBD_OK;
}

// ---------------------------------------------------------------- autotuning
// Time each candidate launch choice for probe width ld on the system's stream
// (CUDA events, one untimed launch then three timed) and keep the fastest.
template <class T> mbd_status autotune_impl(mbd_system *s, int R, int32_t *out) {
    const int ld = probe_ld(R);
    const size_t rows = 3 * (size_t)s->N;
    const size_t npts = (size_t)s->K[0] * s->K[1] * s->K[2];
    PrecData<T> &P = prec<T>(s);
    MBD_TRY(ensure_mesh<T>(s, ld));
    MBD_TRY(s->L.ensure(sizeof(double) * rows * ld));
    MBD_TRY(s->work2.ensure(sizeof(double) * rows * ld));
    MBD_CUDA_TRY(cudaMemsetAsync(P.d.ptr, 0, sizeof(T) * rows * ld, s->stream));
    MBD_CUDA_TRY(cudaMemsetAsync(P.mesh.ptr, 0, sizeof(T) * npts * ld, s->stream));
    MBD_CUDA_TRY(cudaMemsetAsync(s->L.ptr, 0, sizeof(double) * rows * ld, s->stream));
    if (s->real_clusters) MBD_CUDA_TRY(cudaMemsetAsync(P.ereal.ptr, 0, sizeof(T) * rows * ld, s->stream));
    s->tune_ld = ld;
    s->tune_field_apb = s->tune_fft_w = s->tune_sf3_w = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MBD_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaGetLastError();
        return MBD_ERR_CUDA;
    }
    mbd_status st = MBD_OK;
    auto timed = [&](auto &&launch, float *ms) -> mbd_status {
        MBD_TRY(launch());
        MBD_CUDA_TRY(cudaEventRecord(e0, s->stream));
        for (int r = 0; r < 3; ++r) MBD_TRY(launch());
        MBD_CUDA_TRY(cudaEventRecord(e1, s->stream));
        MBD_CUDA_TRY(cudaEventSynchronize(e1));
        MBD_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        return MBD_OK;
    };
    auto run = [&]() -> mbd_status {
        float best = 0.0f, ms = 0.0f;
        if (sizeof(T) == 4) {
            // FFT tile width of every FP32 pass
            int bw = 0;
            for (int w : {32, 16}) {
                s->tune_fft_w = w;
                MBD_TRY(timed([&] { return launch_convolve<T>(s, P.mesh.template as<T>(), ld); }, &ms));
                if (bw == 0 || ms < best) bw = w, best = ms;
            }
            s->tune_fft_w = bw;
            // tile width of the fused spreading + k3 pass
            if (fft_ct_size(s->K[2]) && (ld / 2) % 32 == 0) {
                bw = 0;
                for (int w : {32, 16}) {
                    s->tune_sf3_w = w;
                    MBD_TRY(timed([&] {
                        return launch_spread_fft3<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, ld);
                    }, &ms));
                    if (bw == 0 || ms < best) bw = w, best = ms;
                }
                s->tune_sf3_w = bw;
            }
        }
        // atoms per block of the field kernel
        const int a0 = field_apb(s, ld);
        const int a4 = std::max(1, std::min(64, (s->N + 4 * s->num_sms - 1) / (4 * s->num_sms)));
        std::vector<int> cand = {a0, std::max(1, a0 / 2), std::min(64, 2 * a0), a4};
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        FieldOut<T> fo;
        fo.mode = kFieldApply;
        fo.terms = MBD_TERM_ALL;
        fo.out = s->work2.as<double>();
        fo.xin = s->L.as<double>();
        fo.k = 0;
        std::memset(&fo.lz, 0, sizeof(fo.lz));
        int ba = 0;
        for (int apb : cand) {
            s->tune_field_apb = apb;
            MBD_TRY(timed([&] {
                return launch_field<T>(s, P.d.template as<T>(), P.mesh.template as<T>(), R, ld, fo);
            }, &ms));
            if (ba == 0 || ms < best) ba = apb, best = ms;
        }
        s->tune_field_apb = ba;
        return MBD_OK;
    };
    st = run();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MBD_OK) {
        s->tune_ld = s->tune_field_apb = s->tune_fft_w = s->tune_sf3_w = 0;
        return st;
    }
    if (out) {
        out[0] = ld;
        out[1] = s->tune_field_apb;
        out[2] = s->tune_fft_w;
        out[3] = s->tune_sf3_w;
    }
    return MBD_OK;
}

mbd_status check_run_args(mbd_system *s, int R, int m, double *energy) {
    if (!s || !energy) return MBD_ERR_INVALID_ARG;
    if (R < 1 || R > (1 << 20) || m < 1 || m > kMaxSteps) return MBD_ERR_INVALID_ARG;
    return MBD_OK;
}

}  // namespace
}  // namespace mbd

using namespace mbd;

extern "C" {

const char *mbd_status_string(mbd_status st) {
    switch (st) {
        case MBD_OK: return "MBD_OK";
        case MBD_ERR_INVALID_ARG: return "MBD_ERR_INVALID_ARG";
        case MBD_ERR_OOM: return "MBD_ERR_OOM";
        case MBD_ERR_CUDA: return "MBD_ERR_CUDA";
        case MBD_ERR_NOT_POSITIVE_DEFINITE: return "MBD_ERR_NOT_POSITIVE_DEFINITE";
        case MBD_ERR_NONFINITE: return "MBD_ERR_NONFINITE";
        case MBD_ERR_TIMEOUT: return "MBD_ERR_TIMEOUT";
        case MBD_ERR_UNSUPPORTED: return "MBD_ERR_UNSUPPORTED";
        case MBD_ERR_NO_DEVICE: return "MBD_ERR_NO_DEVICE";
    }
    return "MBD_ERR_UNKNOWN";
}

const char *mbd_last_error(void) { return g_last_error.c_str(); }

mbd_status mbd_set_real_space_method(mbd_system *s, int32_t method) {
    if (!s || method < MBD_REAL_AUTO || method > MBD_REAL_PAIRS) return MBD_ERR_INVALID_ARG;
    if (method == MBD_REAL_CLUSTERS && !s->real_clusters) return MBD_ERR_UNSUPPORTED;
    s->real_method = method;
    return MBD_OK;
}

mbd_status mbd_debug_fail_allocation(int64_t n) {
    g_alloc_countdown.store(n < 0 ? -1 : (long long)n);
    return MBD_OK;
}

mbd_status mbd_create_system(const mbd_system_desc *desc, void *cuda_stream, mbd_system **out) {
    if (out == nullptr) return MBD_ERR_INVALID_ARG;
    MBD_TRY(validate(desc));
    return create_impl(desc, cuda_stream, out);
}

void mbd_destroy_system(mbd_system *sys) {
    if (sys == nullptr) return;
    if (sys->host_scal) cudaFreeHost(sys->host_scal);
    if (sys->host_status) cudaFreeHost(sys->host_status);
    prof_release(sys);
    delete sys;
}

mbd_status mbd_create_batch(int32_t n_sys, const mbd_system_desc *descs, void *cuda_stream, mbd_batch **out) {
    if (out == nullptr || descs == nullptr || n_sys < 1) return MBD_ERR_INVALID_ARG;
    for (int i = 0; i < n_sys; ++i) {
        MBD_TRY(validate(&descs[i]));
        if (descs[i].precision != descs[0].precision) return MBD_ERR_INVALID_ARG;
    }
    mbd_batch *b = new (std::nothrow) mbd_batch();
    if (!b) return MBD_ERR_OOM;
    b->n = n_sys;
    b->precision = descs[0].precision;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    auto fail = [&](mbd_status st) {
        mbd_destroy_batch(b);
        return st;
    };
    cudaError_t ce;
    if ((ce = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess ||
        (ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) {
        set_last_error("batch stream", ce);
        cudaGetLastError();
        return fail(ce == cudaErrorMemoryAllocation ? MBD_ERR_OOM : MBD_ERR_CUDA);
    }
    b->sys.assign(n_sys, nullptr);
    b->streams.assign(n_sys, nullptr);
    b->join.assign(n_sys, nullptr);
    for (int i = 0; i < n_sys; ++i) {
        if ((ce = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking)) != cudaSuccess ||
            (ce = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess) {
            set_last_error("batch member stream", ce);
            cudaGetLastError();
            return fail(MBD_ERR_CUDA);
        }
        const mbd_status st = create_impl(&descs[i], b->streams[i], &b->sys[i]);
        if (st != MBD_OK) {
            b->sys[i] = nullptr;
            return fail(st);
        }
        b->total_atoms += descs[i].n_atoms;
    }
    mbd_status st;
    if ((st = b->seeds_d.ensure(sizeof(uint64_t) * n_sys)) != MBD_OK) return fail(st);
    if ((st = b->out_d.ensure((2 * sizeof(double) + sizeof(int)) * n_sys)) != MBD_OK) return fail(st);
    if (cudaMallocHost(&b->host_seeds, sizeof(uint64_t) * n_sys) != cudaSuccess ||
        cudaMallocHost(&b->host_out, (2 * sizeof(double) + sizeof(int)) * n_sys) != cudaSuccess) {
        cudaGetLastError();
        return fail(MBD_ERR_OOM);
    }
    *out = b;
    return MBD_OK;
}

void mbd_destroy_batch(mbd_batch *b) {
    if (b == nullptr) return;
    destroy_batch_graph(b);
    for (mbd_system *s : b->sys) mbd_destroy_system(s);
    for (cudaStream_t st : b->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->host_seeds) cudaFreeHost(b->host_seeds);
    if (b->host_out) cudaFreeHost(b->host_out);
    delete b;
}

mbd_status mbd_batch_lanczos_energy(mbd_batch *b, int32_t R, int32_t m, const uint64_t *seeds, double *energies,
                                    double *traces, int32_t *failed_member) {
    if (!b || !seeds || !energies) return MBD_ERR_INVALID_ARG;
    if (R < 1 || R > (1 << 20) || m < 1 || m > kMaxSteps) return MBD_ERR_INVALID_ARG;
    if (!b->exec || b->gR != R || b->gm != m) {
        // work queued on the caller's stream before this call precedes the (eager) workspace setup
        MBD_CUDA_TRY(cudaStreamSynchronize(b->stream));
        if (b->precision == MBD_FP64)
            MBD_TRY(capture_batch<double>(b, R, m));
        else
            MBD_TRY(capture_batch<float>(b, R, m));
    }
    const size_t n = (size_t)b->n;
    std::memcpy(b->host_seeds, seeds, sizeof(uint64_t) * n);
    MBD_CUDA_TRY(cudaMemcpyAsync(b->seeds_d.ptr, b->host_seeds, sizeof(uint64_t) * n, cudaMemcpyHostToDevice,
                                 b->stream));
    MBD_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    MBD_CUDA_TRY(cudaMemcpyAsync(b->host_out, b->out_d.ptr, (2 * sizeof(double) + sizeof(int)) * n,
                                 cudaMemcpyDeviceToHost, b->stream));
    MBD_CUDA_TRY(cudaStreamSynchronize(b->stream));
    const double *res = reinterpret_cast<const double *>(b->host_out);
    const int *bits = reinterpret_cast<const int *>(res + 2 * n);
    for (size_t i = 0; i < n; ++i) {
        mbd_status st = status_from_bits(bits[i]);
        if (st == MBD_OK && !std::isfinite(res[2 * i])) st = MBD_ERR_NONFINITE;
        if (st != MBD_OK) {
            if (failed_member) *failed_member = (int32_t)i;
            return st;
        }
    }
    for (size_t i = 0; i < n; ++i) {
        energies[i] = res[2 * i];
        if (traces) traces[i] = res[2 * i + 1];
    }
    return MBD_OK;
}

mbd_status mbd_batch_get_info(const mbd_batch *b, mbd_batch_info *info) {
    if (!b || !info) return MBD_ERR_INVALID_ARG;
    info->n_sys = b->n;
    info->graph_kernels = b->graph_kernels;
    info->total_atoms = b->total_atoms;
    return MBD_OK;
}

mbd_status mbd_autotune(mbd_system *s, int32_t n_probes, int32_t choices[4]) {
    if (!s || n_probes < 1 || n_probes > (1 << 20)) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return autotune_impl<double>(s, n_probes, choices);
    return autotune_impl<float>(s, n_probes, choices);
}

mbd_status mbd_set_launch_choices(mbd_system *s, const int32_t *c) {
    if (!s || !c) return MBD_ERR_INVALID_ARG;
    if (c[0] == 0) {
        s->tune_ld = s->tune_field_apb = s->tune_fft_w = s->tune_sf3_w = 0;
        return MBD_OK;
    }
    const bool fp32 = s->precision != MBD_FP64;
    if (c[0] < 2 || c[0] % 2 != 0 || c[0] > (1 << 20) + 2) return MBD_ERR_INVALID_ARG;
    if (c[1] < 0 || c[1] > 64) return MBD_ERR_INVALID_ARG;
    if (c[2] != 0 && !(fp32 && (c[2] == 16 || c[2] == 32))) return MBD_ERR_INVALID_ARG;
    if (c[3] != 0 && !(fp32 && (c[3] == 16 || c[3] == 32))) return MBD_ERR_INVALID_ARG;
    s->tune_ld = c[0];
    s->tune_field_apb = c[1];
    s->tune_fft_w = c[2];
    s->tune_sf3_w = c[3];
    return MBD_OK;
}

mbd_status mbd_set_basis_storage(mbd_system *s, int32_t mode) {
    if (!s || (mode != MBD_BASIS_STORE && mode != MBD_BASIS_RECOMPUTE)) return MBD_ERR_INVALID_ARG;
    s->basis_recompute = mode == MBD_BASIS_RECOMPUTE ? 1 : 0;
    return MBD_OK;
}

mbd_status mbd_update_positions(mbd_system *s, const double *pos) {
    if (!s || !pos || !finite_all(pos, 3 * (size_t)s->N)) return MBD_ERR_INVALID_ARG;
    wrap_positions(s, pos);
    if (s->precision == MBD_FP64) return setup_geometry<double>(s);
    return setup_geometry<float>(s);
}

mbd_status mbd_apply_C(mbd_system *s, int32_t nvec, const double *x_dev, double *y_dev) {
    if (!s || !x_dev || !y_dev || nvec < 1 || nvec > (1 << 20) || x_dev == y_dev) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return apply_impl<double>(s, nvec, x_dev, y_dev, MBD_TERM_ALL, false);
    return apply_impl<float>(s, nvec, x_dev, y_dev, MBD_TERM_ALL, false);
}

mbd_status mbd_field(mbd_system *s, int32_t nvec, const double *d_dev, double *e_dev, int32_t terms) {
    if (!s || !d_dev || !e_dev || nvec < 1 || nvec > (1 << 20) || d_dev == e_dev) return MBD_ERR_INVALID_ARG;
    if (terms < 0 || terms > MBD_TERM_ALL) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return apply_impl<double>(s, nvec, d_dev, e_dev, terms, true);
    return apply_impl<float>(s, nvec, d_dev, e_dev, terms, true);
}

mbd_status mbd_spread(mbd_system *s, int32_t nvec, const double *d_dev, double *mesh_dev) {
    if (!s || !d_dev || !mesh_dev || nvec < 1 || nvec > (1 << 16)) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return spread_impl<double>(s, nvec, d_dev, mesh_dev);
    return spread_impl<float>(s, nvec, d_dev, mesh_dev);
}

mbd_status mbd_convolve(mbd_system *s, int32_t nvec, const double *in_dev, double *out_dev) {
    if (!s || !in_dev || !out_dev || nvec < 1 || nvec > (1 << 16)) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return convolve_impl<double>(s, nvec, in_dev, out_dev);
    return convolve_impl<float>(s, nvec, in_dev, out_dev);
}

mbd_status mbd_lanczos_energy(mbd_system *s, int32_t R, int32_t m, uint64_t seed, double *energy, double *trace,
                              double *q_host, double *ab_host) {
    MBD_TRY(check_run_args(s, R, m, energy));
    if (s->precision == MBD_FP64) return energy_impl<double>(s, R, m, seed, energy, trace, q_host, ab_host);
    return energy_impl<float>(s, R, m, seed, energy, trace, q_host, ab_host);
}

mbd_status mbd_energy_forces(mbd_system *s, int32_t R, int32_t m, uint64_t seed, double *energy,
                             double *forces_dev) {
    MBD_TRY(check_run_args(s, R, m, energy));
    if (!forces_dev) return MBD_ERR_INVALID_ARG;
    if (s->precision == MBD_FP64) return forces_impl<double>(s, R, m, seed, energy, forces_dev);
    return forces_impl<float>(s, R, m, seed, energy, forces_dev);
}

mbd_status mbd_generate_probes(uint64_t seed, int32_t first, int32_t R, int32_t dim, double *v_dev) {
    if (!v_dev || R < 1 || dim < 1 || first < 0) return MBD_ERR_INVALID_ARG;
    MBD_TRY(launch_probes(seed, first, R, dim, v_dev, nullptr));
    MBD_CUDA_TRY(cudaStreamSynchronize(nullptr));
    return MBD_OK;
}

mbd_status mbd_tridiag_functions(int32_t R, int32_t m, const double *a_host, const double *b_host, int32_t method,
                                 double *q_host, double *c_host) {
    if (!a_host || !b_host || !q_host || R < 1 || m < 1 || m > kMaxSteps) return MBD_ERR_INVALID_ARG;
    if (method != MBD_QUAD_CHEBYSHEV && method != MBD_QUAD_QL && method != MBD_QUAD_QL_DF64)
        return MBD_ERR_INVALID_ARG;
    std::vector<double> a((size_t)m * R), b((size_t)m * R);
    std::vector<int> len(R);
    for (int r = 0; r < R; ++r) {
        int n = m;
        for (int k = 0; k < m - 1; ++k)
            if (b_host[(size_t)r * m + k] == 0.0) {
                n = k + 1;
                break;
            }
        len[r] = n;
        for (int k = 0; k < m; ++k) {
            a[(size_t)k * R + r] = a_host[(size_t)r * m + k];
            b[(size_t)k * R + r] = b_host[(size_t)r * m + k];
        }
    }
    DevBuf da, db, dl, dq, dst, dflag, dc;
    MBD_TRY(da.ensure(sizeof(double) * a.size()));
    MBD_TRY(db.ensure(sizeof(double) * b.size()));
    MBD_TRY(dl.ensure(sizeof(int) * R));
    MBD_TRY(dq.ensure(sizeof(double) * R));
    MBD_TRY(dst.ensure(sizeof(int)));
    MBD_TRY(dflag.ensure(sizeof(int) * R));
    if (c_host) MBD_TRY(dc.ensure(sizeof(double) * a.size()));
    MBD_CUDA_TRY(cudaMemcpy(da.ptr, a.data(), sizeof(double) * a.size(), cudaMemcpyHostToDevice));
    MBD_CUDA_TRY(cudaMemcpy(db.ptr, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice));
    MBD_CUDA_TRY(cudaMemcpy(dl.ptr, len.data(), sizeof(int) * R, cudaMemcpyHostToDevice));
    MBD_CUDA_TRY(cudaMemset(dst.ptr, 0, sizeof(int)));
    MBD_TRY(launch_quadrature(da.as<double>(), db.as<double>(), dl.as<int>(), R, R, m, dq.as<double>(),
                              c_host ? dc.as<double>() : nullptr, dst.as<int>(), dflag.as<int>(), nullptr, method));
    int bits = 0;
    MBD_CUDA_TRY(cudaMemcpy(&bits, dst.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    MBD_TRY(status_from_bits(bits));
    MBD_CUDA_TRY(cudaMemcpy(q_host, dq.ptr, sizeof(double) * R, cudaMemcpyDeviceToHost));
    if (c_host) {
        std::vector<double> c(a.size());
        MBD_CUDA_TRY(cudaMemcpy(c.data(), dc.ptr, sizeof(double) * c.size(), cudaMemcpyDeviceToHost));
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < m; ++k) c_host[(size_t)r * m + k] = c[(size_t)k * R + r];
    }
    return MBD_OK;
}

mbd_status mbd_tridiag_quadrature(int32_t R, int32_t m, const double *a_host, const double *b_host,
                                  double *q_host) {
    return mbd_tridiag_functions(R, m, a_host, b_host, MBD_QUAD_CHEBYSHEV, q_host, nullptr);
}

mbd_status mbd_lanczos_energy_dense(int32_t dim, const double *c_dev, double omega_sum, int32_t R, int32_t m,
                                    uint64_t seed, double *energy, double *q_host, double *ab_host) {
    if (!c_dev || !energy || dim < 1 || R < 1 || m < 1 || m > kMaxSteps) return MBD_ERR_INVALID_ARG;
    // a throwaway system object holds the workspace; no geometry
    mbd_system *s = new (std::nothrow) mbd_system();
    if (!s) return MBD_ERR_OOM;
    s->N = (dim + 2) / 3;
    s->stream = nullptr;
    s->quad_method = MBD_QUAD_CHEBYSHEV;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            s->num_sms = nsm;
        cudaGetLastError();
    }
    s->omega_sum = omega_sum;
    auto run = [&]() -> mbd_status {
        if (cudaMallocHost(&s->host_scal, 16 * sizeof(double)) != cudaSuccess) return MBD_ERR_OOM;
        if (cudaMallocHost(&s->host_status, 4 * sizeof(int)) != cudaSuccess) return MBD_ERR_OOM;
        Lz z;
        MBD_TRY(lanczos_workspace(s, R, m, dim, 1, z));
        MBD_TRY(s->f64.d.ensure(sizeof(double) * (size_t)dim * z.ld));
        MBD_TRY(s->g_d.ensure(sizeof(double) * ((size_t)dim / 3 + 1)));
        // g = 1 so that the prologue's d output is y* itself (unused by the dense operator)
        std::vector<double> ones((size_t)dim / 3 + 1, 1.0);
        MBD_CUDA_TRY(cudaMemcpy(s->g_d.ptr, ones.data(), sizeof(double) * ones.size(), cudaMemcpyHostToDevice));
        // fresh allocations hold whatever the allocator hands back: clear the
        // coefficients and the status word as enqueue_lanczos does
        MBD_CUDA_TRY(cudaMemsetAsync(s->a.ptr, 0, sizeof(double) * (size_t)m * z.ld, s->stream));
        MBD_CUDA_TRY(cudaMemsetAsync(s->b.ptr, 0, sizeof(double) * (size_t)m * z.ld, s->stream));
        MBD_CUDA_TRY(cudaMemsetAsync(s->status.ptr, 0, sizeof(int) * 4, s->stream));
        for (int k = 0; k < m; ++k) {
            MBD_TRY(launch_prologue_t(s->stream, z.v, k, m, seed, R, z.ld, dim, s->g_d.as<double>(), s->f64.d.ptr, 8,
                                      z.nblk));
            MBD_TRY(launch_dense_step(c_dev, dim, z.v, k, R, z.ld, z.nblk, s->stream));
        }
        MBD_TRY(launch_quadrature(z.v.a, z.v.b, z.v.length, R, z.ld, m, s->q.as<double>(), nullptr,
                                  s->status.as<int>(), s->qflag.as<int>(), s->stream, s->quad_method));
        MBD_TRY(launch_energy_reduce(s->q.as<double>(), R, dim, omega_sum, s->scal.as<double>(), s->stream));
        return fetch_results(s, z, energy, nullptr, q_host, ab_host);
    };
    const mbd_status st = run();
    mbd_destroy_system(s);
    return st;
}

mbd_status mbd_profile_enable(mbd_system *s, int32_t enable) {
    if (!s) return MBD_ERR_INVALID_ARG;
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    prof_collect(s);
    for (int k = 0; k < MBD_NUM_STAGES; ++k) {
        s->prof.launches[k] = 0;
        s->prof.ms[k] = 0.0;
    }
    s->prof.timing = enable != 0;
    return MBD_OK;
}

mbd_status mbd_profile_read(mbd_system *s, mbd_profile *out) {
    if (!s || !out) return MBD_ERR_INVALID_ARG;
    MBD_CUDA_TRY(cudaStreamSynchronize(s->stream));
    prof_collect(s);
    out->total_launches = 0;
    for (int k = 0; k < MBD_NUM_STAGES; ++k) {
        out->launches[k] = s->prof.launches[k];
        out->ms[k] = s->prof.ms[k];
        out->total_launches += s->prof.launches[k];
    }
    return MBD_OK;
}

mbd_status mbd_get_info(const mbd_system *s, mbd_info *info) {
    if (!s || !info) return MBD_ERR_INVALID_ARG;
    info->n_atoms = s->N;
    for (int a = 0; a < 3; ++a) info->mesh[a] = s->K[a];
    info->n_pairs = s->nnz;
    info->precision = s->precision;
    long long bytes = 0;
    const DevBuf *bufs[] = {&s->pos_d, &s->g_d, &s->w2_d, &s->rvdw_d, &s->row_d, &s->col_d, &s->shift_d,
                            &s->top_d, &s->bin_start_d, &s->bin_atoms_d, &s->order_d, &s->Y, &s->L, &s->a, &s->b,
                            &s->invb, &s->length, &s->partial, &s->counter, &s->q, &s->scal, &s->status, &s->work, &s->wacc, &s->v0,
                            &s->work2, &s->f64.pairA, &s->f64.w, &s->f64.dw, &s->f64.d2w, &s->f64.G, &s->f64.d,
                            &s->f64.mesh, &s->f32.pairA, &s->f32.w, &s->f32.dw, &s->f32.d2w, &s->f32.G, &s->f32.d,
                            &s->f32.mesh};
    for (const DevBuf *b : bufs) bytes += (long long)b->bytes;
    info->device_bytes = bytes;
    return MBD_OK;
}

}  // extern "C"
