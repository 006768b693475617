// Internal declarations shared by the translation units of libmbd.
//
// Data layout on the device (probe-innermost, "ld" = padded probe count, even):
//   Lanczos vectors (FP64)      [3N][ld]           row (3i + alpha), column = probe
//   dipoles d, fields E (T)     [N][3][ld]         same indexing as above
//   SPME mesh (T)               [K1][K2][K3][ld]   = complex [K1][K2][K3][ld/2]:
//                               probes (2v, 2v+1) form the real/imaginary parts
//                               of one complex vector; since the influence
//                               function is real and even, one complex FFT
//                               convolution serves two probes exactly.
//   spline stencil (T)          w, dw [N][3][p]    M_p(frac(u) + t), M_p'(...), t = 0..p-1
//                               for mesh points top - t (mod K) per dimension
//   real-space pairs            CSR over atoms i: col j, packed image shift,
//                               pair tensor A (6 unique entries xx xy xz yy yz zz)
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "mbd.h"

namespace mbd {

constexpr int kMaxSteps = 128;
constexpr int kMaxOrder = 10;
constexpr int kMaxRadixStages = 12;
constexpr double kBreakdown = 1e-14;

template <class T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };

// ---------------------------------------------------------------- errors
void set_last_error(const char *where, cudaError_t e);
#define MBD_CUDA_TRY(call)                                               \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) {                                         \
            ::mbd::set_last_error(#call, e_);                            \
            return e_ == cudaErrorMemoryAllocation ? MBD_ERR_OOM : MBD_ERR_CUDA; \
        }                                                                \
    } while (0)
#define MBD_LAUNCH_CHECK() MBD_CUDA_TRY(cudaGetLastError())

// Programmatic dependent launch in a Lanczos step: a kernel launched with it
// may be scheduled while its predecessor in the stream runs its last blocks.
// The kernels of the step let their successor launch at once
// (pdl_launch_dependents, their first instruction) and wait for their
// predecessor's completion and memory (pdl_wait) before they touch global
// data.  The successor launches only when every block of the predecessor has
// started, so its early blocks take resources only from the predecessor's
// tail.  Both instructions are no-ops in a kernel launched without the
// attribute.  Measured per kernel: early launch helps the fused spreading
// (after the prologue) and the FFT passes while the mesh fits in L2; it slows
// the FFT passes on meshes beyond L2, and the prologue and field kernels at
// every size, which are therefore launched plainly.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(bool early, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = early ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args &&>(args)...);
}
#define MBD_TRY(expr)                       \
    do {                                    \
        mbd_status s_ = (expr);             \
        if (s_ != MBD_OK) return s_;        \
    } while (0)

// ---------------------------------------------------------------- device buffer
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    mbd_status ensure(size_t n);   // grow (contents not preserved)
    void release();
    template <class U> U *as() const { return static_cast<U *>(ptr); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
};

// ---------------------------------------------------------------- kernel argument blocks
struct Geom {
    int N;
    int K1, K2, K3;
    int p;
    double cmat[9];     // C[beta*3+alpha] = K_beta a*_{beta, alpha} (du_beta / dR_alpha)
    double cell[9];
};

template <class T> struct SplineView {
    const int *top;     // [N][3] floor(u) in [0, K)
    const T *w;         // [N][3][p]
    const T *dw;        // [N][3][p]
    const T *d2w;       // [N][3][p] (forces only)
};

// Cell grid of the neighbour search (built on the host, searched on the device).
struct NeighborGrid {
    int N;
    int nc[3], kk[3];       // cells per direction; cells searched each way
    const int *start;       // [ncell + 1]
    const int *atoms;       // [N] atoms by cell
    const int *cidx;        // [N][3] cell coordinates of each atom
    double cell[9];
    double r2max;
};

struct BinView {
    int nb1, nb2, nb3;      // bricks (= bins) per dimension
    int bs1, bs2, bs3;      // brick edge (mesh points)
    int nc1, nc2, nc3;      // candidate bins per dimension for one brick
    const int *start;       // [nbins+1]
    const int *atoms;       // [N] atoms sorted by bin
};

template <class T> struct PairView {
    const int *row;     // [N+1]
    const int *col;     // [nnz]
    const int *shift;   // [nnz] packed (n1+128) | (n2+128)<<8 | (n3+128)<<16
    const T *A;         // [nnz][6]
};

struct LanczosView {
    double *Y;          // [yslots][3N][ld] basis, y_k in slot k mod yslots (y* written by the
                        // prologue, y after the field kernel); yslots = m, or 3 when the basis
                        // is recomputed instead of stored
    double *L;          // [3N][ld] l_k = C y_k
    double *a;          // [m][ld]
    double *b;          // [m][ld]  b[k] couples y_k and y_{k+1}
    double *invb;       // [ld]     1/b for the current step (0 after breakdown)
    int *length;        // [ld]     Krylov length per probe (m unless broken down)
    double *partial;    // [nblk][ld] block partial sums
    double *gpartial;   // [ngroups][ld] group sums (two-level reduction)
    unsigned *counter;  // [nchunk][cstride] last-block counters (self-resetting)
    int cstride;        // counters per probe chunk (>= ngroups + 1)
    int yslots;
    double *W;          // [3N][ld] when set: the field kernel adds coef[k] y_k (recomputed basis)
    const double *coef; // [m][ld] c = Delta^{-1/2} e_1, read with W
};
__host__ __device__ inline size_t lz_slot(const LanczosView &lz, int k) { return (size_t)(k % lz.yslots); }

// Deterministic two-level reduction across the blocks of a grid row
// (blockIdx.y = probe chunk).  Each block contributes bval[t] for the probes
// rbase + t (t < nloc); blocks are grouped by kRedGroup; the last block of a
// group sums its group in block order, the last group finisher sums the groups
// in group order.  Returns true (block-uniformly) in exactly one block, whose
// out[t] then holds the grid totals.  Counters reset themselves.
constexpr int kRedGroup = 16;
__device__ __forceinline__ bool grid_reduce(const double *bval, int nloc, int rbase, int R, int ld,
                                            const LanczosView &lz, double *out) {
    __shared__ bool s_last;
    const int t = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const unsigned nblk = gridDim.x;
    const unsigned ngroups = (nblk + kRedGroup - 1) / kRedGroup;
    unsigned *cnt = lz.counter + (size_t)blockIdx.y * lz.cstride;
    for (int k = t; k < nloc; k += nthr)
        if (rbase + k < R) lz.partial[(size_t)blockIdx.x * ld + rbase + k] = bval[k];
    __threadfence();
    __syncthreads();
    const unsigned g = blockIdx.x / kRedGroup;
    const unsigned gsize = min((unsigned)kRedGroup, nblk - g * kRedGroup);
    if (t == 0) s_last = (atomicAdd(&cnt[g], 1u) == gsize - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int k = t; k < nloc; k += nthr) {
        const int r = rbase + k;
        if (r < R) {
            double s = 0.0;
            for (unsigned b = g * kRedGroup; b < g * kRedGroup + gsize; ++b) s += __ldcg(&lz.partial[(size_t)b * ld + r]);
            lz.gpartial[(size_t)g * ld + r] = s;
        }
    }
    if (t == 0) cnt[g] = 0u;
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = (atomicAdd(&cnt[ngroups], 1u) == ngroups - 1);
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    for (int k = t; k < nloc; k += nthr) {
        const int r = rbase + k;
        double s = 0.0;
        if (r < R)
            for (unsigned gg = 0; gg < ngroups; ++gg) s += __ldcg(&lz.gpartial[(size_t)gg * ld + r]);
        out[k] = s;
    }
    if (t == 0) cnt[ngroups] = 0u;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- per-system state
struct SystemData;

// One nonzero of the transposed stencil matrix: the Cartesian weights
// dW_j(k)/dR_j of atom j at mesh point k (row = k).  For float the atom index
// travels in the .w component (bit pattern), for double in a separate word.
template <class T> struct SpreadRec;
template <> struct __align__(16) SpreadRec<float> { float w0, w1, w2; int atom; };
template <> struct __align__(16) SpreadRec<double> { double w0, w1, w2; int atom; int pad; };

// One (pencil, atom) record of the factorised spreading: for the pencil
// (k1, k2) and an atom j whose stencil covers it (t1 = top1 - k1, t2 = top2 - k2
// mod K), the weights along the pencil are
//   dW_j/dR_alpha (k1, k2, top3 - t3) = M3(t3) e0_alpha + M3'(t3) e1_alpha,
//   e0_alpha = C_{0 alpha} M1'(t1) M2(t2) + C_{1 alpha} M1(t1) M2'(t2),
//   e1_alpha = C_{2 alpha} M1(t1) M2(t2),   C_{beta alpha} = K_beta a*_{beta alpha}.
// Records are grouped by the mesh point (k1, k2, top3_j) (CSR over points).
// Clusters of the real-space field: kClusterSize consecutive atoms of the
// Morton order; a cluster with more than kClusterSortCap pairs in all (more
// than 256 neighbours per atom on average) sends the system back to the
// per-atom pair loop of the field kernel.
constexpr int kClusterSize = 16;
constexpr int kClusterSortCap = 4096;
// One real-space pair of a cluster atom: the index of the neighbour entry
// within the cluster and the pair tensor A (xx xy xz yy yz zz).
template <class T> struct __align__(16) RealPair {
    int e;
    int pad;
    T a[6];
};

constexpr int kPencilOrder = 6;   // the spline order the pencil spreading is compiled for
template <class T> struct __align__(16) PencilRec {
    T e0[3], e1[3];
    int atom, top3;
};

template <class T> struct PrecData {
    DevBuf pairA;       // [nnz][6]
    DevBuf pairdA;      // [nnz][18] dA_ab/dr_c (forces)
    DevBuf srow;        // [K^3 + 1] CSR row pointers of the spread matrix
    DevBuf srec;        // [216 N] SpreadRec<T>
    DevBuf prow;        // [K^3 + 1] CSR over points (k1, k2, top3) of the pencil records (spline order 6)
    DevBuf prec;        // [36 N] PencilRec<T>
    DevBuf k3w;         // [N][16] M3(t3) (t3 < p) at 0.., M3'(t3) at 8..
    DevBuf w, dw, d2w;  // [N][3][p]
    DevBuf G;           // [K1K2K3] influence function
    DevBuf tw1, tw2, tw3;   // twiddles [K] complex per dimension
    DevBuf cA;          // [nnz] RealPair<T>: per (cluster, atom), sorted by entry (real-space clusters)
    DevBuf ereal;       // [N][3][ld] real-space field of the current dipoles (cluster kernel output)
    DevBuf d;           // dipoles [N][3][ld]
    DevBuf mesh;        // [K1K2K3][ld]
};

// Stage profiler: launch counts always, CUDA-event timing when enabled.
struct Profiler {
    bool timing = false;
    long long launches[MBD_NUM_STAGES] = {};
    double ms[MBD_NUM_STAGES] = {};
    struct Rec {
        int stage;
        cudaEvent_t e0, e1;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
};

struct FFTDim {
    int K;
    int nst;
    int radix[kMaxRadixStages];
};

}  // namespace mbd

struct mbd_system {
    // parameters
    int N;
    double cell[9], recip[9], volume;
    int K[3], p;
    double ewald_beta, r_cut, damp_cut, damp_beta, damp_d;
    int precision;
    int quad_method;    // MBD_QUAD_*: Chebyshev quadrature (QL fallback) or QL
    int num_sms = 1;    // multiprocessors of the device the system lives on
    // launch choices made by mbd_autotune or mbd_set_launch_choices for probe
    // width tune_ld (0: the built-in rules): field-kernel atoms per block, FP32
    // FFT and fused-spreading tiles
    int tune_ld = 0, tune_field_apb = 0, tune_fft_w = 0, tune_sf3_w = 0;
    int basis_recompute = 0;    // MBD_BASIS_RECOMPUTE: three basis vectors kept, the forces rerun the recurrence
    cudaStream_t stream;
    double omega_sum;
    mbd::FFTDim fft[3];
    // host copies
    std::vector<double> pos, alpha, omega, rvdw;
    // common device data
    mbd::DevBuf pos_d, g_d, w2_d, rvdw_d;            // [N][3], [N], [N], [N]
    mbd::DevBuf row_d, col_d, shift_d;              // CSR
    mbd::DevBuf cell_start_d, cell_atoms_d, cell_idx_d, nb_err_d;   // neighbour-search cell grid
    mbd::DevBuf top_d;                              // [N][3]
    mbd::DevBuf w64_d, dw64_d;                      // [N][3][p] FP64 stencil weights (setup)
    mbd::DevBuf bin_start_d, bin_atoms_d, order_d;  // spread bins; field atom order
    mbd::DevBuf bin_of_d, bin_cursor_d;             // [N] brick of each atom, [nbins] fill cursors
    mbd::DevBuf morton_cnt, morton_start;           // Morton order of the bricks (setup scratch)
    // real-space clusters: the distinct neighbours j of each cluster (CSR by
    // cluster) and the pair starts per (cluster, atom) [8 nclus + 1]
    mbd::DevBuf cl_ecnt, cl_pcnt, cl_estart, cl_pstart, cl_entries, cl_err;
    int n_clusters = 0;
    bool real_clusters = false;                     // the clusters of the last geometry were built
    int real_method = MBD_REAL_AUTO;                // mbd_set_real_space_method
    mbd::DevBuf scan_cnt, scan_bsum;                // count / scan scratch of the geometry setup
    long long nb_cap = 0;   // pairs col_d, shift_d and the pair tensors hold (0: not sized yet)
    mbd::NeighborGrid ngrid{};   // the last neighbour search's grid
    mbd::BinView bins;
    long long nnz;
    // precision-specific
    mbd::PrecData<double> f64;
    mbd::PrecData<float> f32;
    // Lanczos workspace
    mbd::DevBuf Y, L, a, b, invb, length, partial, gpartial, counter, q, scal, status, work, work2;
    mbd::DevBuf qflag;          // [ld] probes the Chebyshev quadrature hands to QL
    mbd::DevBuf wacc, v0;       // recomputed basis: w = sum_k c_k y_k and y_0
    int counter_stride = 0;
    mbd::DevBuf forces_acc;
    mbd::Profiler prof;
    // pinned host staging
    double *host_scal = nullptr;
    int *host_status = nullptr;
};

namespace mbd {

// ---------------------------------------------------------------- launchers (kernels_*.cu)
// setup
// Atoms binned by the brick of their top stencil point (B's geometry), in
// increasing atom index within a brick: counts, starts [nbins + 1], atoms [N].
mbd_status launch_bin_atoms(int N, const int *top, const BinView &B, int *bin_of, int *cnt, int *start,
                            int *cursor, int *atoms, DevBuf &bsum, cudaStream_t st);
// fill: writes the pairs below cap only (the caller compares row[N] with cap)
mbd_status launch_neighbors(const NeighborGrid &ng, const double *pos, int *cnt_or_row, int *col, int *shift,
                            int *err, bool fill, long long cap, cudaStream_t st);
mbd_status launch_exclusive_scan(const int *in, int *out, int n, DevBuf &bsum, cudaStream_t st);
template <class T> mbd_status launch_pair_tensors(mbd_system *s, cudaStream_t st);
mbd_status launch_morton_order(const BinView &B, int N, int *order, DevBuf &cnt, DevBuf &start, DevBuf &bsum,
                               cudaStream_t st);
template <class T>
mbd_status launch_cluster_pairs(mbd_system *s, const int *order, int nclus, DevBuf &ecnt, DevBuf &pcnt,
                                DevBuf &estart, DevBuf &pstart, DevBuf &entries, DevBuf &A, int *err,
                                cudaStream_t st);
// whether this call's real-space field runs on the clusters (probe width ld)
bool real_on_clusters(const mbd_system *s, int ld, int real_bytes);
// E_real = sum over real-space pairs A d_j of the clusters (T [N][3][ld])
template <class T> mbd_status launch_real_clusters(mbd_system *s, const T *d, T *ereal, int ld, cudaStream_t st);
template <class T> mbd_status launch_splines(mbd_system *s, cudaStream_t st);
template <class T> mbd_status launch_influence(mbd_system *s, const double *bmod_host, cudaStream_t st);

// mesh stages
template <class T> mbd_status launch_spread(mbd_system *s, const T *d, T *mesh, int R, int ld);
template <class T> mbd_status build_spread_matrix(mbd_system *s);
// in place; skip_first: the forward k3 pass was already done (launch_spread_fft3)
template <class T> mbd_status launch_convolve(mbd_system *s, T *mesh, int ld, bool skip_first = false);
template <class T> mbd_status launch_spread_fft3(mbd_system *s, const T *d, T *mesh, int R, int ld);
bool spread_fft3_supported(const mbd_system *s, int ld, int real_bytes);
bool fft_ct_size(int K);        // a compile-time FFT pass exists for this length
enum FieldMode { kFieldOut = 0, kFieldApply = 1, kFieldLanczos = 2 };
template <class T> struct FieldOut {
    int mode;
    int terms;
    double *out;            // kFieldOut: E [3N][ld]; kFieldApply: y [3N][ld]
    const double *xin;      // kFieldApply: x [3N][ld]
    LanczosView lz;         // kFieldLanczos
    int k;                  // Lanczos step
};
template <class T> mbd_status launch_field(mbd_system *s, const T *d, const T *mesh, int R, int ld,
                                           const FieldOut<T> &o);

// Lanczos
mbd_status launch_prologue_t(cudaStream_t st, const LanczosView &lz, int k, int m, uint64_t seed, int R, int ld,
                             int rows, const double *g, void *dout, int dtype_bytes, int nblk,
                             const uint64_t *seed_dev = nullptr);
// Quadrature of every probe's tridiagonal, q [R] and, when coef != nullptr,
// c = Delta^{-1/2} e_1 as coef [m][ld]: MBD_QUAD_CHEBYSHEV (default) runs the
// Chebyshev kernel and QL for the probes it flags in fallback [ld]; the QL methods
// run QL for all.
mbd_status launch_quadrature(const double *a, const double *b, const int *length, int R, int ld, int m, double *q,
                             double *coef, int *status, int *fallback, cudaStream_t st, int method);
mbd_status launch_energy_reduce(const double *q, int R, int dim, double omega_sum, double *scal, cudaStream_t st);
mbd_status launch_probes(uint64_t seed, int first, int R, int dim, double *v, cudaStream_t st);
mbd_status launch_dense_step(const double *c, int dim, const LanczosView &lz, int k, int R, int ld, int nblk,
                             cudaStream_t st);
int field_vec(int ld, int real_bytes);
bool field_half(int ld, int real_bytes);
int field_apb(const mbd_system *s, int ld);
int field_blocks(const mbd_system *s, int ld);

// layout helpers
mbd_status launch_to_probe_major(const double *x, int nvec, int rows, double *xt, int ld, cudaStream_t st);
mbd_status launch_from_probe_major(const double *xt, int nvec, int rows, int ld, double *x, cudaStream_t st);
template <class T> mbd_status launch_cast_rows(const double *x, T *y, size_t n, cudaStream_t st);
template <class T> mbd_status launch_mesh_out(const T *mesh, int nvec, size_t npts, int ld, double *out,
                                              cudaStream_t st);
template <class T> mbd_status launch_mesh_in(const double *in, int nvec, size_t npts, int ld, T *mesh,
                                             cudaStream_t st);

// forces
template <class T>
mbd_status launch_force_dipoles_w_t(mbd_system *s, const double *w, const double *v, int R, int ld, T *dpq,
                                    int ld2);
template <class T>
mbd_status launch_force_dipoles_t(mbd_system *s, const double *Y, const double *coef, const int *length, int R,
                                  int ld, int m, T *dpq, int ld2);
template <class T>
mbd_status launch_force_gather_t(mbd_system *s, const T *dpq, const T *mesh, int R, int ld2, double scale,
                                 double *forces);

// misc
int probe_ld(int R);
void prof_begin(mbd_system *s, int stage, cudaEvent_t *e0);
void prof_end(mbd_system *s, int stage, int n_launches, cudaEvent_t e0);
void prof_release(mbd_system *s);
#define MBD_STAGE(s, stage, nl, call)                       \
    do {                                                   \
        cudaEvent_t ev0_ = nullptr;                        \
        ::mbd::prof_begin((s), (stage), &ev0_);            \
        mbd_status st_ = (call);                           \
        ::mbd::prof_end((s), (stage), (nl), ev0_);         \
        if (st_ != MBD_OK) return st_;                     \
    } while (0)

}  // namespace mbd
