// Internal declarations of libesi (not part of the C ABI).
//
// Discrete scheme shared by every propagation kernel (forward and adjoint):
//   new = cur + gamma (cur - old) + alpha * cc * (L(cur) + dx^2 src)
// with L the dimensionless 8th-order Laplacian sum (Lap8 u = L / dx^2), cc = v^2 dt^2 / dx^2,
// alpha = 1 / (1 + kappa), gamma = (1 - kappa) / (1 + kappa), kappa = eta dt / 2 the
// sponge coefficient.  This is the centred discretisation of
//   (1/v^2)(u_tt + eta u_t) - Lap u = q,
// rearranged from (1+kappa) u_{n+1} = 2 u_n - (1-kappa) u_{n-1} + c (Lap8 u_n + q_n).
//
// The adjoint uses the same kernel run backward in time: the blocks of the discrete
// operator A = C^{-1} M (C = diag(c), M the block lower-triangular time-stepping
// matrix) are spatially symmetric, so A^T is A with the time axis reversed, and
// S^T e = A^{-T} R^T e is the same recurrence driven by R^T e from t = T down to 0.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is fetched through the runtime at run time)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "esi.h"

namespace esi {

// ----------------------------------------------------------------------------- tiling
constexpr int HALO = 4;             // stencil radius (8th order)
constexpr int TX2 = 64;             // tile width (x) of the 2D step kernel
#ifndef ESI_TZ2
#define ESI_TZ2 32
#endif
constexpr int TZ2 = ESI_TZ2;        // tile height (z)
constexpr int NT2 = 256;            // threads per block of the 2D step kernel
constexpr int SW2 = TX2 + 2 * HALO; // shared tile width incl. halo (72: 16-byte rows)
constexpr int SH2 = TZ2 + 2 * HALO; // shared tile height incl. halo
constexpr int MAXP = 8;             // interpolation points per receiver (4 in 2D, 8 in 3D)
constexpr int PITCH = 32;           // x pitch multiple of the state / internal arrays

// 3D kernel tile (xy plane, marching along z)
constexpr int TX3 = 32, TY3 = 16;
constexpr int SW3 = TX3 + 2 * HALO, SH3 = TY3 + 2 * HALO;
// z chunks: each block marches one chunk of planes; the chunk count of a context is chosen
// at creation (step3_chunks) so that the grid fills whole waves of resident blocks, with
// chunks of ZCH3_MIN .. ZCH3_MAX planes
constexpr int ZCH3_MIN = 40, ZCH3_MAX = 100;
constexpr int RING3 = 8;            // staged planes (shared-memory ring of TMA boxes)
constexpr int DFT_BLOCK = 16;       // shortest block of a blocked DTFT pass (steps)

// first plane of z chunk zc when nz planes are split into nzc chunks of near-equal length
__host__ __device__ inline int chunk_begin3(int zc, int nzc, int nz) {
    return (int)((long long)zc * nz / nzc);
}

// ----------------------------------------------------------------------------- feature flags
enum : unsigned {
    F_EXT = 1u << 0,  // add a dense extended source field q_n
    F_CGP = 1u << 1,  // source p' = r + beta p (CG direction update), written back to p
    F_PT = 1u << 2,   // point injection (wavelet at sources, or R^T e at receivers)
    F_SMP = 1u << 3,  // sample the *input* state into a trace buffer
    F_OUT = 1u << 4,  // write the new state to a dense space-time output
    F_AP = 1u << 5,   // CG product epilogue Ap = new + beta B^2 p and <p, Ap> partials
    F_STW = 1u << 6,  // write the stash s = L + dx^2 q (gradient recompute)
    F_GRD = 1u << 7,  // gradient: G += new * stash
    F_SAD = 1u << 8,  // saddle-point gradient: G += B^2 q s
    F_DFT = 1u << 9,  // on-the-fly DTFT: the new state into the block stash (slot slot_w)
};

// Point lists on the device, CSR over (shot, tile).  Injection lists hold unique nodes
// with their contributing traces; sampling lists hold receivers with MAXP points each.
template <typename T>
struct InjList {
    const int *tile_ptr = nullptr;     // [ns * ntiles + 1]
    const int *cell = nullptr;         // [nodes] local cell index inside the tile (no halo)
    const int *cptr = nullptr;         // [nodes + 1] range into contributions
    const long long *off0 = nullptr;   // [contribs] trace offset at time 0
    const int *tstride = nullptr;      // [contribs] trace stride per time step
    const T *w = nullptr;              // [contribs] weight (dx^2 folded in)
};

template <typename T>
struct SmpList {
    const int *tile_ptr = nullptr;     // [ns * ntiles + 1]
    const int *idx = nullptr;          // [recs * MAXP] shared-tile index (incl. halo)
    const long long *gidx = nullptr;   // [recs * MAXP] global index into a shot's state
    const T *w = nullptr;              // [recs * MAXP]
    const long long *off0 = nullptr;   // [recs] output offset at time 0
    const int *tstride = nullptr;      // [recs]
    const int *shot = nullptr;         // [recs] shot of each receiver
    int nrec = 0;
};

// Layouts.  States and every internal field (CG vectors, stash, accumulators) are pitched:
// plane = nz * ny * px elements, x pitch px = round_up(nx, 32), pad columns zero.  Fields
// owned by the caller (extended sources, adjoint outputs) are dense: plane N = nz*ny*nx.
template <typename T>
struct StepArgs {
    CUtensorMap tm;            // TMA map of the input state: 2D box (SW2, SH2, 1), 3D box
                               // (SW3, SH3, 1, 1) (one tile with its halo)
    CUtensorMap tm_old;        // the older state, tile-interior box (3D; 2D CG product)
    CUtensorMap tm_cc;         // c = v^2 dt^2 / dx^2, tile-interior box (3D; 2D CG product)
    int *dev_err;              // sticky device error word (bounded waits that gave up)
    int nz, ny, nx, px;        // grid and pitch (elements) of the state arrays
    long long sst;             // pitched plane (= shot stride of state arrays)
    long long N;               // dense plane nz*ny*nx
    long long fst;             // shot stride of dense caller space-time fields (nt * N)
    long long fstp;            // shot stride of internal pitched space-time fields (nt * sst)
    int opx;                   // row pitch of the F_OUT target (nx: caller, px: internal)
    long long oplane, ofst;    // its plane and shot strides
    int ntx, nty, ntz;         // tiles per shot
    const T *cur;              // input state
    T *po;                     // in: older state, out: new state
    const T *cc;               // [nz][ny][px] v^2 dt^2 / dx^2
    const T *kz, *ky, *kx;     // sponge kappa per row / column
    T dx2;
    int n;                     // time index of dense sources (ext / CG / stash slot base)
    const int *active;         // per-shot flag or null
    // extended source at time n: ext + s*fst + n*N
    const T *ext;
    // CG: r, p at time n
    const T *cg_r;
    T *cg_p;
    const double *cg_beta;
    int cg_first;
    T cg_pc;                   // > 0: diagonal preconditioner z = r * ipb2 in p' = z + beta p
    // per-shot maps [ns][sst] (pitched) of pen B^2 and 1 / (pen B^2), B = |x - x_s| + eps
    const T *pb2, *ipb2;
    // learned preconditioner: z = r * ipb2 + y[(s*ng + n/16)][iz/2][ix/2][n%16] (FP32)
    const float *pc_y;         // learned preconditioner: time-sample planes of its correction
    const double *pc_theta;    // and its per-shot weight
    int pc_ng, pc_hc, pc_wc;
    // point injection at trace time tin
    InjList<T> inj;
    const T *inj_trace;
    int tin;
    // sampling of the input state at trace time tout (skipped when tout < 0)
    SmpList<T> smp;
    T *smp_out;
    int tout;
    // output of the new state at time nout: fout + s*ofst + nout*oplane + row*opx + x
    T *fout;
    int nout;
    // CG product (internal pitched): ap/ap_p at time nout; <p,Ap> block partials per shot
    T *ap;
    const T *ap_p;
    double *dot_part;
    T pen;                     // penalty beta
    const double *src_pos;     // [ns][3] source (x, y, z) metres
    T eps, dx;
    int unit_b;                // F_SAD: the annihilator is the identity (WRI), not ||x - x_s|| + eps
    // stash [slot][ns][sst] pitched; write slot sw, read slot sr
    T *stash_w;
    const T *stash_r;
    int slot_w, slot_r, ns;
    // gradient accumulators [ns][sst] pitched
    T *grad;
    // DTFT: twiddles [nt][nf][2] (cos, sin) of the new state's time; acc [ns][nf][sst][2]
    int nf;
    const T *twid;
    T *dft;
};

// device error codes written to StepArgs::dev_err
constexpr int DEV_ERR_TMA_TIMEOUT = 1;
// iteration limit of the mbarrier wait for a TMA tile (a tile arrives in microseconds;
// the limit is seconds of polling)
constexpr long long TMA_WAIT_LIMIT = 1ll << 26;

// ----------------------------------------------------------------------------- launchers
template <typename T>
cudaError_t launch_step2(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st,
                         bool chained = false);
template <typename T>
cudaError_t launch_step3(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st,
                         bool chained);
// number of z chunks for a 3D context: cols = x tiles * y tiles * shots, element size esz
// (the resident blocks per SM of the step kernel on the current device enter the choice)
int step3_chunks(int nz, long long cols, int esz);

// sample a whole state (global memory) for every receiver of a list at time tout
template <typename T>
cudaError_t launch_sample_global(const SmpList<T> &l, const T *state, long long sst, T *out,
                                 int tout, cudaStream_t st);

// c = v^2 dt^2 / dx^2 into a pitched array; per-block max |v| partials
template <typename T>
cudaError_t launch_setup_cc(const T *v, T *cc, int nz, int ny, int nx, int px, double dt,
                            double dx, double *vmax_part, int nblk, cudaStream_t st);

// per-shot reductions of dense [ns][len] vectors into block partials [ns][nblk]
template <typename T>
cudaError_t launch_dot(const T *a, const T *b, long long len, long long sstride, int ns,
                       double *part, int nblk, const int *active, cudaStream_t st);
cudaError_t launch_reduce_partials(const double *part, int nblk, int ns, double *out,
                                   cudaStream_t st);

// x += alpha p (x dense caller layout) ; r -= alpha Ap (pitched) ; partial ||r||^2.
// rows = nt * nz * ny rows of nx cells per shot; r, p, Ap rows have pitch px.
// With ipb2 (per-shot [sst] map of 1 / (pen B^2)) also the partial r^T z, z = r * ipb2.
template <typename T>
cudaError_t launch_cg_update(T *x, T *r, const T *p, const T *ap, long long rows, int nx, int px,
                             int ns, const double *alpha, const int *active, double *part,
                             double *part2, int nblk, const T *ipb2, long long sst, int nzny,
                             cudaStream_t st);

// per-shot maps pb2 = pen B^2 and ipb2 = 1 / pb2 over the pitched plane (pad cells 0); with
// unit_b the annihilator is the identity (WRI: pb2 = pen)
template <typename T>
cudaError_t launch_b2_maps(T *pb2, T *ipb2, int ns, int nz, int ny, int nx, int px, T pen, T eps,
                           T dx, const double *src_pos, int unit_b, cudaStream_t st);
// y = x - y over len elements
template <typename T>
cudaError_t launch_sub_from(T *y, const T *x, long long len, cudaStream_t st);
// out = the sum of G consecutive partial vectors of length n (in order)
template <typename T>
cudaError_t launch_sum_parts(T *out, const T *parts, int G, long long n, cudaStream_t st);
// data-space CG vectors (traces layout; shot s owns [seg[s], seg[s+1])), partials [ns][64]:
// ap = p + kp in place over kp with <p, ap>; x += alpha p, r -= alpha ap with ||r||^2; p = r + beta p
constexpr int DVEC_NBLK = 64;
template <typename T>
cudaError_t launch_dvec_ident_dot(T *kp, const T *p, const long long *seg, const int *active,
                                  double *part, int ns, cudaStream_t st);
template <typename T>
cudaError_t launch_dvec_update(T *x, T *r, const T *p, const T *ap, const long long *seg,
                               const double *alpha, const int *active, double *part, int ns,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_dvec_xpby(T *p, const T *r, const long long *seg, const double *beta,
                             const int *active, int ns, cudaStream_t st);
// q[s][t][N] (dense) = f[s][t][pitched] * ipb2[s][pitched]
template <typename T>
cudaError_t launch_scale_to_dense(T *q, const T *f, const T *ipb2, int ns, int nt, int rows,
                                  int nx, int px, long long sst, cudaStream_t st);
// alpha = rr / pAp ; flags breakdown
cudaError_t launch_cg_alpha(const double *rr, const double *pap, double *alpha, int *bad,
                            const int *active, int ns, cudaStream_t st);
// out += pen B^2 p over dense caller fields [ns][nt][N]
template <typename T>
cudaError_t launch_add_b2p(T *out, const T *p, int ns, int nt, int nz, int ny, int nx, T pen, T eps,
                           T dx, const double *src_pos, cudaStream_t st);
// beta = rr_new / rr_old ; rr_old = rr_new
cudaError_t launch_cg_beta(double *rr_old, const double *rr_new, double *beta,
                           const int *active, int ns, cudaStream_t st);

// misfit: e = d - dobs (in place into d), per-block partial 1/2 e^2
template <typename T>
cudaError_t launch_residual(T *d, const T *dobs, long long len, double *part, int nblk,
                            cudaStream_t st);

// gradient finalisation: g[i] = scale_i * sum_s G[s][i]  (G pitched [ns][sst], g dense)
template <typename T>
cudaError_t launch_grad_finalize(const T *G, int ns, long long sst, const T *cc, int nz, int ny,
                                 int nx, int px, double dt, double dx, double extra, int param,
                                 T *g, cudaStream_t st);

// Two-level checkpoint codec (FP16 / BF16): coarse part = the even-index cells, fine part =
// the residual against their multilinear interpolation, each with a per-shot scale (vec.cu).
// With `sub` non-null the encoder codes u - sub; with `base` non-null the decoder stores
// base - x.  `bits` holds 2 ns words of scratch.
long long ckpt_coarse_size(int nz, int ny, int nx);
template <typename T>
cudaError_t launch_ckpt_encode(const T *u, const T *sub, int ns, int nz, int ny, int nx, int px,
                               long long sst, int kind, unsigned *bits, uint16_t *fine,
                               uint16_t *coarse, float *fscale, float *cscale, cudaStream_t st);
template <typename T>
cudaError_t launch_ckpt_decode(const uint16_t *fine, const uint16_t *coarse, const float *fscale,
                               const float *cscale, int ns, int nz, int ny, int nx, int px,
                               long long sst, int kind, const T *base, T *u, cudaStream_t st);

// Blocked DTFT: a context stashes the new states of DFT_BLOCK_MAX, 32 or DFT_BLOCK steps at a
// time, the longest block whose stash fits its budget (dft_block_steps); longer blocks read
// and write the accumulators less often.
constexpr int DFT_BLOCK_MAX = 64;
int dft_block_steps(long long stash_plane_bytes, size_t device_bytes);

// Blocked DTFT: acc [ns][nf][sst][2] += sum_k snap[k][ns][sst] (cos, sin)(twid[k][nf]) over the
// K <= DFT_BLOCK_MAX stashed states of one block.  Rows of px cells of which nx are real:
// 16-byte chunks that lie wholly in the pad are skipped (the step kernels never write them,
// so the stash holds whatever the memory held there; the accumulators keep their zero pads).
template <typename T>
cudaError_t launch_dft_block(const T *snap, int K, int ns, long long sst, int nx, int px, int nf,
                             const T *twid, T *acc, cudaStream_t st);

// Frequency-domain ESI (Eq. "idtft", "normaldtft"), at most FD_MAXF frequencies.
constexpr int FD_MAXF = 8;
// inverse DTFT of one block: src[s][k][cell] = sum_m re(qb_m) tw[k][m].x + im(qb_m) tw[k][m].y
// for the K <= kst steps of the block (kst slots per shot), qb pitched complex slices
// [ns][nf][sst][2]
template <typename T>
cudaError_t launch_idft_block(const T *qb, int K, int kst, int ns, long long sst, int nf,
                              const T *tw, T *src, cudaStream_t st);
// out_m += pb2 * sum_m' G[m][m'] p_m' per cell (G = F F^H / nt, complex [nf][nf][2]) and the
// per-block partials of Re <p, out> ([ns][DVEC_NBLK]); inactive shots skipped
template <typename T>
cudaError_t launch_fd_b2g_dot(T *out, const T *p, const T *pb2, const double *G, int nf, int ns,
                              long long sst, const int *active, double *part, cudaStream_t st);

// Objective and outer loop: per-shot partials [ns][nblk] of 1/2 sum pb2 q^2 over the dense
// field q[ns][nt][rows * nx]; dense model-vector dot and max |a| partials [nblk];
// z = alpha x + beta y (y may be NULL), clamped to [lo, hi] when lo < hi
template <typename T>
cudaError_t launch_penalty(const T *q, const T *pb2, int ns, int nt, long long rows, int nx,
                           int px, long long sst, double *part, int nblk, cudaStream_t st);
template <typename T>
cudaError_t launch_mdot(const T *a, const T *b, long long n, double *part, int nblk,
                        cudaStream_t st);
template <typename T>
cudaError_t launch_mamax(const T *a, long long n, double *part, int nblk, cudaStream_t st);
template <typename T>
cudaError_t launch_mlincomb(T *z, double alpha, const T *x, double beta, const T *y, long long n,
                            double lo, double hi, cudaStream_t st);

// z = w r per cell at every frequency of the complex slices [ns][nf][sst][2] (w per shot
// [ns][sst]) with the partials of Re <r, z> ([ns][DVEC_NBLK]); inactive shots skipped
template <typename T>
cudaError_t launch_fd_precond(T *z, const T *r, const T *w, int nf, int ns, long long sst,
                              const int *active, double *part, cudaStream_t st);

// DTFT output: pitched accumulators [ns][nf][sst][2] -> caller dense [ns][nf][N][2], either
// copied in the field precision (half == 0) or as half pairs with a per (shot, f) scale
template <typename T>
cudaError_t launch_dft_output(const T *acc, long long sst, int rows, int nx, int px, int ns,
                              int nf, int half, void *out, unsigned *absmax_bits,
                              float *scales_dev, cudaStream_t st);

}  // namespace esi

#include <atomic>

namespace esi {

// A launch setting worked out once per device (a kernel's shared-memory attribute, its
// resident blocks per SM): function attributes belong to each device's context, so a process
// that drives several devices sets them on each.  Thread-safe; 0 means "not yet computed".
struct PerDevice {
    static constexpr int MAXDEV = 64;
    std::atomic<int> v[MAXDEV];
};

// *out = the cached value for the current device, computing it with compute(int *) on the
// first call there (a failing compute is returned and retried on the next call)
template <typename Fn>
cudaError_t per_device(PerDevice &c, int *out, Fn &&compute) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= PerDevice::MAXDEV) return cudaErrorInvalidDevice;
    int v = c.v[dev].load(std::memory_order_acquire);
    if (v == 0) {
        if ((e = compute(&v)) != cudaSuccess) return e;
        c.v[dev].store(v, std::memory_order_release);
    }
    *out = v;
    return cudaSuccess;
}

}  // namespace esi
