// Streaming kernels around the propagators: model set-up, per-shot reductions with a
// deterministic two-stage sum, the CG vector updates of Algorithm 1, misfit, gradient
// finalisation, and the scaled FP16/BF16 snapshot codec.
#include "esi_internal.h"

namespace esi {
namespace {

constexpr int RT = 256;  // threads per block of the streaming kernels

template <typename T>
struct alignas(16) V16 {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum in double; result valid in thread 0
__device__ __forceinline__ double block_sum_d(double v) {
    __shared__ double red[RT / 32];
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < RT / 32 ? red[lane] : 0.0;
        t = warp_sum_d(t);
    }
    return t;
}

template <typename T>
__global__ void setup_cc_kernel(const T *v, T *cc, int nz, int ny, int nx, int px, double dt,
                                double dx, double *vmax_part) {
    const long long N = (long long)nz * ny * nx;
    const double s = dt * dt / (dx * dx);
    double vm = 0.0;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < N;
         i += (long long)gridDim.x * RT) {
        const long long row = i / nx, x = i - row * nx;
        const double vv = double(v[i]);
        cc[row * px + x] = T(vv * vv * s);
        vm = fmax(vm, fabs(vv));
    }
    __shared__ double red[RT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vm = fmax(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RT / 32; ++w) t = fmax(t, red[w]);
        vmax_part[blockIdx.x] = t;
    }
}

// <a, b> per shot over pitched vectors (len a multiple of the 16-byte vector width; pad
// elements are zero): 16-byte loads, a field-precision sum per vector, double across.
template <typename T>
__global__ void dot_kernel(const T *a, const T *b, long long len, long long sstride,
                           double *part, const int *active) {
    constexpr int VEC = V16<T>::n;
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const V16<T> *x = reinterpret_cast<const V16<T> *>(a + s * sstride);
    const V16<T> *y = reinterpret_cast<const V16<T> *>(b + s * sstride);
    double acc = 0.0;
    const long long nv = len / VEC;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < nv;
         i += (long long)gridDim.x * RT) {
        const V16<T> u = x[i], w = y[i];
        T t = T(0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) t += u.v[k] * w.v[k];
        acc += double(t);
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
}

__global__ void reduce_partials_kernel(const double *part, int nblk, int ns, double *out) {
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += RT) acc += part[(long long)s * nblk + i];
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) out[s] = t;
}

// Algorithm 1's vector updates for one shot per blockIdx.y: x_{k+1} = x_k + alpha p_k
// (x in the caller's dense layout), r_{k+1} = r_k - alpha A p_k (pitched), with the
// partial ||r_{k+1}||^2 and, for the diagonal preconditioner z = r / (pen B^2), r^T z.
template <typename T>
__global__ void cg_update_kernel(T *x, T *r, const T *p, const T *ap, long long rows, int nx,
                                 int px, const double *alpha, const int *active, double *part,
                                 double *part2, const T *ipb2, long long sst, int nzny) {
    constexpr int VEC = V16<T>::n;
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const T al = T(alpha[s]);
    const long long sp = rows * px, sd = rows * nx;   // shot strides (pitched, dense)
    T *xs = x + s * sd;
    T *rs = r + s * sp;
    const T *ps = p + s * sp, *as = ap + s * sp;
    const int cpr = px / VEC;
    const long long nchunk = rows * cpr;
    const T *ib = ipb2 ? ipb2 + s * sst : nullptr;
    double acc = 0.0, acc2 = 0.0;
    for (long long c = (long long)blockIdx.x * RT + threadIdx.x; c < nchunk;
         c += (long long)gridDim.x * RT) {
        const long long row = c / cpr;
        const int x0 = int(c - row * cpr) * VEC;
        if (x0 >= nx) continue;
        const long long pi = row * px + x0;
        const V16<T> pv = *reinterpret_cast<const V16<T> *>(ps + pi);
        const V16<T> av = *reinterpret_cast<const V16<T> *>(as + pi);
        V16<T> rv = *reinterpret_cast<const V16<T> *>(rs + pi);
        T t = T(0);
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            rv.v[k] -= al * av.v[k];
            t += rv.v[k] * rv.v[k];
        }
        *reinterpret_cast<V16<T> *>(rs + pi) = rv;
        T *xr = xs + row * nx + x0;
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if (x0 + k < nx) xr[k] += al * pv.v[k];
        acc += double(t);
        if (ib) {   // r^T z with z = r / (pen B^2)
            const V16<T> bv = *reinterpret_cast<const V16<T> *>(ib + (row % nzny) * px + x0);
            T t2 = T(0);
#pragma unroll
            for (int k = 0; k < VEC; ++k) t2 += rv.v[k] * rv.v[k] * bv.v[k];
            acc2 += double(t2);
        }
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
    if (ib) {
        __syncthreads();
        const double t2 = block_sum_d(acc2);
        if (threadIdx.x == 0) part2[(long long)s * gridDim.x + blockIdx.x] = t2;
    }
}

__global__ void cg_alpha_kernel(const double *rr, const double *pap, double *alpha, int *bad,
                                const int *active, int ns) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    if (active && !active[s]) {
        alpha[s] = 0.0;
        return;
    }
    const double a = rr[s] / pap[s];
    if (!(pap[s] > 0.0) || !isfinite(a)) {
        bad[s] = 1;
        alpha[s] = 0.0;
    } else {
        alpha[s] = a;
    }
}

__global__ void cg_beta_kernel(double *rr_old, const double *rr_new, double *beta,
                               const int *active, int ns) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    if (active && !active[s]) return;
    beta[s] = rr_new[s] / rr_old[s];
    rr_old[s] = rr_new[s];
}

// ---- data-space CG vectors: one flat traces-layout array, shot s owning [seg[s], seg[s+1])
// ap = p + kp (in place over kp) with per-shot partials of <p, ap>
template <typename T>
__global__ void dvec_ident_dot_kernel(T *kp, const T *p, const long long *seg, const int *active,
                                      double *part) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    double acc = 0.0;
    for (long long i = seg[s] + (long long)blockIdx.x * RT + threadIdx.x; i < seg[s + 1];
         i += (long long)gridDim.x * RT) {
        const T a = p[i] + kp[i];
        kp[i] = a;
        acc += double(p[i]) * double(a);
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
}

// x += alpha p, r -= alpha ap, per-shot partials of ||r||^2
template <typename T>
__global__ void dvec_update_kernel(T *x, T *r, const T *p, const T *ap, const long long *seg,
                                   const double *alpha, const int *active, double *part) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const T al = T(alpha[s]);
    double acc = 0.0;
    for (long long i = seg[s] + (long long)blockIdx.x * RT + threadIdx.x; i < seg[s + 1];
         i += (long long)gridDim.x * RT) {
        x[i] += al * p[i];
        const T rv = r[i] - al * ap[i];
        r[i] = rv;
        acc += double(rv) * double(rv);
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
}

// p = r + beta p
template <typename T>
__global__ void dvec_xpby_kernel(T *p, const T *r, const long long *seg, const double *beta,
                                 const int *active) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const T b = T(beta[s]);
    for (long long i = seg[s] + (long long)blockIdx.x * RT + threadIdx.x; i < seg[s + 1];
         i += (long long)gridDim.x * RT)
        p[i] = r[i] + b * p[i];
}

// q[s][t][cell] (caller dense) = f[s][t][pitched cell] * ipb2[s][pitched cell]
template <typename T>
__global__ void scale_to_dense_kernel(T *q, const T *f, const T *ipb2, int nt, int rows, int nx,
                                      int px, long long sst) {
    const int s = blockIdx.y;
    const long long N = (long long)rows * nx, len = N * nt;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < len;
         i += (long long)gridDim.x * RT) {
        const long long t = i / N, c = i - t * N;
        const long long row = c / nx;
        const long long pc = row * px + (c - row * nx);
        q[(long long)s * len + i] = f[((long long)s * nt + t) * sst + pc] * ipb2[(long long)s * sst + pc];
    }
}

template <typename T>
__global__ void sub_from_kernel(T *y, const T *x, long long len) {
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < len;
         i += (long long)gridDim.x * RT)
        y[i] = x[i] - y[i];
}

template <typename T>
__global__ void residual_kernel(T *d, const T *dobs, long long len, double *part) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < len;
         i += (long long)gridDim.x * RT) {
        const T e = d[i] - dobs[i];
        d[i] = e;
        acc += double(e) * double(e);
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = 0.5 * t;
}

template <typename T>
__global__ void grad_finalize_kernel(const T *G, int ns, long long N, long long sst,
                                     const T *cc, int nx, int px, double dt, double dx,
                                     double extra, int param, T *g) {
    const double dx2 = dx * dx;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < N;
         i += (long long)gridDim.x * RT) {
        const long long row = i / nx, x = i - row * nx;
        const long long pi = row * px + x;
        double sum = 0.0;
        for (int s = 0; s < ns; ++s) sum += double(G[(long long)s * sst + pi]);
        const double c = double(cc[pi]) * dx2;  // v^2 dt^2
        double gc = extra * sum / (c * dx2);
        if (param == ESI_PARAM_V) gc *= 2.0 * sqrt(c) * dt;
        else if (param == ESI_PARAM_M) gc *= -(c * c) / (dt * dt);
        g[i] = T(gc);
    }
}

// ---------------------------------------------------------------- snapshot codec
constexpr float CODEC_RANGE = 32768.0f;  // max |u| of a snapshot maps to this magnitude

// Two-level checkpoint code.  A snapshot x (a wave state, or with `sub` the difference
// u_n - u_{n-1}) is stored as
//   coarse: x at the cells whose indices are all even, [ns][ncz][ncy][ncx] dense;
//   fine  : x - U(coarse) at every cell, in the pitched state layout (pad cells 0);
// each part in FP16 or BF16, U the multilinear interpolation between even cells of the
// decoded coarse part (an odd index averages its two even neighbours, the last one repeats
// its left neighbour).  Rounding then leaves an error of the format's precision relative
// to the interpolation residual, which is a small fraction of x for fields resolved by
// several cells per wavelength, instead of relative to x itself: the Laplacian of the
// recomputed states sees far less rounding noise.  The encoder forms the residual against
// the decoded coarse part, so the decoder reproduces x to the fine part's rounding.  FP16
// parts carry a per-shot scale (max |part| -> CODEC_RANGE, for FP16's narrow exponent
// range); BF16 has the exponent range of FP32 and is stored unscaled (scale 1).
// The fine and decode kernels give each thread 8 cells of a row (16-byte loads and stores);
// the coarse kernel walks the rows of the even cells.
struct CkDims {
    int nz, ny, nx, px;
    int ncz, ncy, ncx;
    long long sst, csst;   // per-shot sizes of the fine (pitched) and coarse (dense) parts
};

__device__ __forceinline__ float ck_dec(uint16_t c, int kind) {
    return kind == ESI_CKPT_F16 ? __half2float(__ushort_as_half(c))
                                : __bfloat162float(__ushort_as_bfloat16(c));
}

__device__ __forceinline__ uint16_t ck_enc(float y, int kind) {
    return kind == ESI_CKPT_F16 ? __half_as_ushort(__float2half_rn(y))
                                : __bfloat16_as_ushort(__float2bfloat16_rn(y));
}

// The coarse rows that row (z, y) interpolates from: (z0, y0), (z0, y1), (z1, y0), (z1, y1),
// where an odd index takes its even neighbours (the last one its left one twice) and an even
// one its own row; zo / yo: whether the second row along z / y enters the mean.
struct CkRows {
    const uint16_t *r00, *r01, *r10, *r11;
    bool zo, yo;
};

__device__ __forceinline__ CkRows ck_rows(const uint16_t *cs, const CkDims &d, int z, int y) {
    const int z0 = z >> 1, z1 = (z & 1) ? min(z0 + 1, d.ncz - 1) : z0;
    const int y0 = y >> 1, y1 = (y & 1) ? min(y0 + 1, d.ncy - 1) : y0;
    CkRows c;
    c.r00 = cs + ((long long)z0 * d.ncy + y0) * d.ncx;
    c.r01 = cs + ((long long)z0 * d.ncy + y1) * d.ncx;
    c.r10 = cs + ((long long)z1 * d.ncy + y0) * d.ncx;
    c.r11 = cs + ((long long)z1 * d.ncy + y1) * d.ncx;
    c.zo = (z & 1) != 0;
    c.yo = (y & 1) != 0;
    return c;
}

// Cells per thread of the fine and decode kernels: 16 bytes of codes, 16-byte loads of the
// state (rows are px = a multiple of 32 cells long, so chunks never straddle rows).
constexpr int CK_CH = 8;

// U(coarse) at the CK_CH cells x0 .. x0 + 7 of a row (x0 a multiple of 8), in T, the same
// arithmetic in the encoder and the decoder: the decoded coarse values of columns
// x0/2 .. x0/2 + 4 (clamped to the last column) summed over the row's coarse rows; an even
// cell takes its column's mean, an odd one the mean of its two columns.
template <typename T>
__device__ __forceinline__ void ck_interp8(const CkRows &c, float cscale, const CkDims &d, int x0,
                                           int kind, T out[CK_CH]) {
    const int k0 = x0 >> 1;
    T col[CK_CH / 2 + 1];
#pragma unroll
    for (int j = 0; j <= CK_CH / 2; ++j) {
        const int k = min(k0 + j, d.ncx - 1);
        T acc = T(ck_dec(c.r00[k], kind) * cscale);
        if (c.yo) acc += T(ck_dec(c.r01[k], kind) * cscale);
        if (c.zo) {
            acc += T(ck_dec(c.r10[k], kind) * cscale);
            if (c.yo) acc += T(ck_dec(c.r11[k], kind) * cscale);
        }
        col[j] = acc;
    }
    const int n = (c.zo ? 2 : 1) * (c.yo ? 2 : 1);
    const T w1 = T(1.0 / n), w2 = T(0.5 / n);
#pragma unroll
    for (int m = 0; m < CK_CH / 2; ++m) {
        out[2 * m] = col[m] * w1;
        out[2 * m + 1] = (col[m] + col[m + 1]) * w2;
    }
}

// CK_CH consecutive values of a state (16-byte aligned)
template <typename T>
__device__ __forceinline__ void ck_load8(const T *p, T v[CK_CH]) {
#pragma unroll
    for (int h = 0; h < CK_CH / V16<T>::n; ++h) {
        const V16<T> t = reinterpret_cast<const V16<T> *>(p)[h];
#pragma unroll
        for (int i = 0; i < V16<T>::n; ++i) v[h * V16<T>::n + i] = t.v[i];
    }
}

template <typename T>
__device__ __forceinline__ T ck_value(const T *u, const T *sub, long long i) {
    return sub ? u[i] - sub[i] : u[i];
}

// the coarse part: pass 0 max |x| over the even cells (FP16 only), pass 1 the codes
template <typename T>
__global__ void ck_coarse_kernel(const T *u, const T *sub, CkDims d, int pass, int kind,
                                 unsigned *bits, uint16_t *coarse, float *cscale) {
    const int s = blockIdx.y;
    const T *x = u + s * d.sst;
    const T *y = sub ? sub + s * d.sst : nullptr;
    float inv = 1.0f;
    if (pass == 1 && kind == ESI_CKPT_F16) {
        const float mx = __uint_as_float(bits[s]);
        inv = mx > 0.0f ? __fdiv_rn(CODEC_RANGE, mx) : 0.0f;
        if (blockIdx.x == 0 && threadIdx.x == 0) cscale[s] = __fdiv_rn(mx, CODEC_RANGE);
    } else if (pass == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        cscale[s] = 1.0f;
    }
    uint16_t *cs = coarse + s * d.csst;
    float m = 0.0f;
    for (int row = blockIdx.x; row < d.ncz * d.ncy; row += gridDim.x) {
        const int cz = row / d.ncy, cy = row - cz * d.ncy;
        const long long src = ((long long)(2 * cz) * d.ny + 2 * cy) * d.px;
        for (int cx = threadIdx.x; cx < d.ncx; cx += blockDim.x) {
            const float v = float(ck_value(x, y, src + 2 * cx));
            if (pass == 0)
                m = fmaxf(m, fabsf(v));
            else
                cs[(long long)row * d.ncx + cx] = ck_enc(kind == ESI_CKPT_F16 ? __fmul_rn(v, inv) : v, kind);
        }
    }
    if (pass == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // non-negative floats order like their bit patterns
        if ((threadIdx.x & 31) == 0) atomicMax(bits + s, __float_as_uint(m));
    }
}

// the fine part: pass 0 max |x - U(coarse)| (FP16 only), pass 1 the codes (pads 0); a thread
// takes CK_CH cells of a row at a time
template <typename T>
__global__ void ck_fine_kernel(const T *u, const T *sub, CkDims d, int pass, int kind,
                               unsigned *bits, const uint16_t *coarse, const float *cscale,
                               uint16_t *fine, float *fscale) {
    const int s = blockIdx.y;
    const T *x = u + s * d.sst;
    const T *y = sub ? sub + s * d.sst : nullptr;
    const uint16_t *cs = coarse + s * d.csst;
    const float sc = cscale[s];
    float inv = 1.0f;
    if (pass == 1 && kind == ESI_CKPT_F16) {
        const float mx = __uint_as_float(bits[s]);
        inv = mx > 0.0f ? __fdiv_rn(CODEC_RANGE, mx) : 0.0f;
        if (blockIdx.x == 0 && threadIdx.x == 0) fscale[s] = __fdiv_rn(mx, CODEC_RANGE);
    } else if (pass == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        fscale[s] = 1.0f;
    }
    uint16_t *fs = fine + s * d.sst;
    const int cpr = d.px / CK_CH;   // chunks per row
    const long long nch = (long long)d.nz * d.ny * cpr;
    float m = 0.0f;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nch;
         q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / cpr;
        const int x0 = (int)(q - row * cpr) * CK_CH;
        const long long base = row * d.px + x0;
        uint16_t code[CK_CH];
#pragma unroll
        for (int i = 0; i < CK_CH; ++i) code[i] = 0;
        if (x0 < d.nx) {
            const int z = (int)(row / d.ny), yy = (int)(row - (long long)z * d.ny);
            T ip[CK_CH], xv[CK_CH], yv[CK_CH];
            ck_interp8<T>(ck_rows(cs, d, z, yy), sc, d, x0, kind, ip);
            ck_load8<T>(x + base, xv);
            if (y) ck_load8<T>(y + base, yv);
#pragma unroll
            for (int i = 0; i < CK_CH; ++i) {
                if (x0 + i >= d.nx) continue;   // pad cells: code 0
                const float v = float((y ? xv[i] - yv[i] : xv[i]) - ip[i]);
                if (pass == 0)
                    m = fmaxf(m, fabsf(v));
                else
                    code[i] = ck_enc(kind == ESI_CKPT_F16 ? __fmul_rn(v, inv) : v, kind);
            }
        }
        if (pass == 1) {
            uint4 w;
            w.x = code[0] | ((unsigned)code[1] << 16);
            w.y = code[2] | ((unsigned)code[3] << 16);
            w.z = code[4] | ((unsigned)code[5] << 16);
            w.w = code[6] | ((unsigned)code[7] << 16);
            *reinterpret_cast<uint4 *>(fs + base) = w;
        }
    }
    if (pass == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(bits + s, __float_as_uint(m));
    }
}

// x = U(coarse) + fine; with `base`, u_{n-1} = base - x (base holds the decoded u_n); a thread
// takes CK_CH cells of a row at a time
template <typename T>
__global__ void ck_decode_kernel(const uint16_t *fine, const uint16_t *coarse,
                                 const float *fscale, const float *cscale, CkDims d, int kind,
                                 const T *base, T *u) {
    const int s = blockIdx.y;
    const uint16_t *cs = coarse + s * d.csst;
    const uint16_t *fs = fine + s * d.sst;
    const float sc = cscale[s], sf = fscale[s];
    T *x = u + s * d.sst;
    const T *b = base ? base + s * d.sst : nullptr;
    const int cpr = d.px / CK_CH;
    const long long nch = (long long)d.nz * d.ny * cpr;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nch;
         q += (long long)gridDim.x * blockDim.x) {
        const long long row = q / cpr;
        const int x0 = (int)(q - row * cpr) * CK_CH;
        const long long off = row * d.px + x0;
        T v[CK_CH];
#pragma unroll
        for (int i = 0; i < CK_CH; ++i) v[i] = T(0);   // pad columns stay zero
        if (x0 < d.nx) {
            const int z = (int)(row / d.ny), yy = (int)(row - (long long)z * d.ny);
            T ip[CK_CH], bv[CK_CH];
            ck_interp8<T>(ck_rows(cs, d, z, yy), sc, d, x0, kind, ip);
            const uint4 w = *reinterpret_cast<const uint4 *>(fs + off);
            const unsigned wd[4] = {w.x, w.y, w.z, w.w};
            if (b) ck_load8<T>(b + off, bv);
#pragma unroll
            for (int i = 0; i < CK_CH; ++i) {
                if (x0 + i >= d.nx) continue;
                const uint16_t code = (uint16_t)(wd[i >> 1] >> ((i & 1) * 16));
                const T t = ip[i] + T(__fmul_rn(ck_dec(code, kind), sf));
                v[i] = b ? bv[i] - t : t;
            }
        }
#pragma unroll
        for (int h = 0; h < CK_CH / V16<T>::n; ++h) {
            V16<T> o;
#pragma unroll
            for (int i = 0; i < V16<T>::n; ++i) o.v[i] = v[h * V16<T>::n + i];
            reinterpret_cast<V16<T> *>(x + off)[h] = o;
        }
    }
}

// DTFT accumulators: pitched [ns*nf][sst][2] (pad cells zero) -> caller dense [ns*nf][N][2]
template <typename T>
__global__ void dft_absmax_kernel(const T *acc, long long sst, unsigned *bits) {
    const int sm = blockIdx.y;  // shot * nf + m
    const T *a = acc + (long long)sm * sst * 2;
    float m = 0.0f;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < 2 * sst;
         i += (long long)gridDim.x * RT)
        m = fmaxf(m, fabsf(float(a[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(bits + sm, __float_as_uint(m));
}

template <typename T>
__global__ void dft_out_kernel(const T *acc, long long sst, int rows, int nx, int px, int half,
                               const unsigned *bits, void *out, float *scales) {
    const int sm = blockIdx.y;
    const long long N = (long long)rows * nx;
    float inv = 1.0f;
    if (half) {
        const float mx = __uint_as_float(bits[sm]);
        inv = mx > 0.0f ? __fdiv_rn(CODEC_RANGE, mx) : 0.0f;
        if (blockIdx.x == 0 && threadIdx.x == 0) scales[sm] = __fdiv_rn(mx, CODEC_RANGE);
    }
    const T *a = acc + (long long)sm * sst * 2;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < N;
         i += (long long)gridDim.x * RT) {
        const long long row = i / nx, x = i - row * nx;
        const long long pi = (row * px + x) * 2;
        const long long o = ((long long)sm * N + i) * 2;
        if (half) {
            __half *h = reinterpret_cast<__half *>(out);
            h[o] = __float2half_rn(__fmul_rn(float(a[pi]), inv));
            h[o + 1] = __float2half_rn(__fmul_rn(float(a[pi + 1]), inv));
        } else {
            T *d = reinterpret_cast<T *>(out);
            d[o] = a[pi];
            d[o + 1] = a[pi + 1];
        }
    }
}

inline int blocks_for(long long len, int cap) {
    long long b = (len + RT - 1) / RT;
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace

template <typename T>
cudaError_t launch_setup_cc(const T *v, T *cc, int nz, int ny, int nx, int px, double dt,
                            double dx, double *vmax_part, int nblk, cudaStream_t st) {
    setup_cc_kernel<T><<<nblk, RT, 0, st>>>(v, cc, nz, ny, nx, px, dt, dx, vmax_part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dot(const T *a, const T *b, long long len, long long sstride, int ns,
                       double *part, int nblk, const int *active, cudaStream_t st) {
    dot_kernel<T><<<dim3(nblk, ns), RT, 0, st>>>(a, b, len, sstride, part, active);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const double *part, int nblk, int ns, double *out,
                                   cudaStream_t st) {
    reduce_partials_kernel<<<ns, RT, 0, st>>>(part, nblk, ns, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cg_update(T *x, T *r, const T *p, const T *ap, long long rows, int nx, int px,
                             int ns, const double *alpha, const int *active, double *part,
                             double *part2, int nblk, const T *ipb2, long long sst, int nzny,
                             cudaStream_t st) {
    cg_update_kernel<T><<<dim3(nblk, ns), RT, 0, st>>>(x, r, p, ap, rows, nx, px, alpha, active,
                                                       part, part2, ipb2, sst, nzny);
    return cudaGetLastError();
}

template <typename T>
__global__ void add_b2p_kernel(T *out, const T *p, int nt, int nz, int ny, int nx, T pen, T eps,
                               T dx, const double *src_pos) {
    const int s = blockIdx.y;
    const long long N = (long long)nz * ny * nx, len = N * nt;
    const double xs = src_pos[3 * s], ys = src_pos[3 * s + 1], zs = src_pos[3 * s + 2];
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < len;
         i += (long long)gridDim.x * RT) {
        const long long c = i % N;
        const int ix = int(c % nx);
        const long long row = c / nx;
        const int iy = int(row % ny), iz = int(row / ny);
        const double ex = ix * double(dx) - xs, ez = iz * double(dx) - zs;
        const double ey = ny > 1 ? iy * double(dx) - ys : 0.0;
        const double B = std::sqrt(ex * ex + ey * ey + ez * ez) + double(eps);
        out[(long long)s * len + i] += T(double(pen) * B * B) * p[(long long)s * len + i];
    }
}

template <typename T>
__global__ void b2_maps_kernel(T *pb2, T *ipb2, int nz, int ny, int nx, int px, T pen, T eps,
                               T dx, const double *src_pos, int unit_b) {
    const int s = blockIdx.y;
    const long long plane = (long long)nz * ny * px;
    const double xs = src_pos[3 * s], ys = src_pos[3 * s + 1], zs = src_pos[3 * s + 2];
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < plane;
         i += (long long)gridDim.x * RT) {
        const long long row = i / px;
        const int x = int(i - row * px);
        const int iy = int(row % ny), iz = int(row / ny);
        T v = T(0), iv = T(0);
        if (x < nx) {
            const double ex = x * double(dx) - xs, ez = iz * double(dx) - zs;
            const double ey = ny > 1 ? iy * double(dx) - ys : 0.0;
            const double B = unit_b ? 1.0 : std::sqrt(ex * ex + ey * ey + ez * ez) + double(eps);
            v = T(double(pen) * B * B);
            iv = T(1.0 / (double(pen) * B * B));
        }
        pb2[(long long)s * plane + i] = v;
        if (ipb2) ipb2[(long long)s * plane + i] = iv;
    }
}

template <typename T>
cudaError_t launch_add_b2p(T *out, const T *p, int ns, int nt, int nz, int ny, int nx, T pen, T eps,
                           T dx, const double *src_pos, cudaStream_t st) {
    const long long len = (long long)nz * ny * nx * nt;
    add_b2p_kernel<T><<<dim3(blocks_for(len, 4096), ns), RT, 0, st>>>(out, p, nt, nz, ny, nx, pen,
                                                                      eps, dx, src_pos);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_b2_maps(T *pb2, T *ipb2, int ns, int nz, int ny, int nx, int px, T pen, T eps,
                           T dx, const double *src_pos, int unit_b, cudaStream_t st) {
    const long long plane = (long long)nz * ny * px;
    b2_maps_kernel<T><<<dim3(blocks_for(plane, 2048), ns), RT, 0, st>>>(pb2, ipb2, nz, ny, nx, px,
                                                                        pen, eps, dx, src_pos, unit_b);
    return cudaGetLastError();
}

cudaError_t launch_cg_alpha(const double *rr, const double *pap, double *alpha, int *bad,
                            const int *active, int ns, cudaStream_t st) {
    cg_alpha_kernel<<<(ns + 127) / 128, 128, 0, st>>>(rr, pap, alpha, bad, active, ns);
    return cudaGetLastError();
}

cudaError_t launch_cg_beta(double *rr_old, const double *rr_new, double *beta,
                           const int *active, int ns, cudaStream_t st) {
    cg_beta_kernel<<<(ns + 127) / 128, 128, 0, st>>>(rr_old, rr_new, beta, active, ns);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dvec_ident_dot(T *kp, const T *p, const long long *seg, const int *active,
                                  double *part, int ns, cudaStream_t st) {
    dvec_ident_dot_kernel<T><<<dim3(DVEC_NBLK, ns), RT, 0, st>>>(kp, p, seg, active, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dvec_update(T *x, T *r, const T *p, const T *ap, const long long *seg,
                               const double *alpha, const int *active, double *part, int ns,
                               cudaStream_t st) {
    dvec_update_kernel<T><<<dim3(DVEC_NBLK, ns), RT, 0, st>>>(x, r, p, ap, seg, alpha, active, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dvec_xpby(T *p, const T *r, const long long *seg, const double *beta,
                             const int *active, int ns, cudaStream_t st) {
    dvec_xpby_kernel<T><<<dim3(DVEC_NBLK, ns), RT, 0, st>>>(p, r, seg, beta, active);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_to_dense(T *q, const T *f, const T *ipb2, int ns, int nt, int rows,
                                  int nx, int px, long long sst, cudaStream_t st) {
    scale_to_dense_kernel<T><<<dim3(blocks_for((long long)rows * nx * nt, 4096), ns), RT, 0, st>>>(
        q, f, ipb2, nt, rows, nx, px, sst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sub_from(T *y, const T *x, long long len, cudaStream_t st) {
    sub_from_kernel<T><<<blocks_for(len, 4096), RT, 0, st>>>(y, x, len);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(T *d, const T *dobs, long long len, double *part, int nblk,
                            cudaStream_t st) {
    residual_kernel<T><<<nblk, RT, 0, st>>>(d, dobs, len, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_grad_finalize(const T *G, int ns, long long sst, const T *cc, int nz, int ny,
                                 int nx, int px, double dt, double dx, double extra, int param,
                                 T *g, cudaStream_t st) {
    const long long N = (long long)nz * ny * nx;
    grad_finalize_kernel<T><<<blocks_for(N, 8192), RT, 0, st>>>(G, ns, N, sst, cc, nx, px, dt, dx,
                                                                extra, param, g);
    return cudaGetLastError();
}

CkDims ck_dims(int nz, int ny, int nx, int px, long long sst) {
    CkDims d;
    d.nz = nz, d.ny = ny, d.nx = nx, d.px = px;
    d.ncz = (nz + 1) / 2, d.ncy = (ny + 1) / 2, d.ncx = (nx + 1) / 2;
    d.sst = sst;
    d.csst = (long long)d.ncz * d.ncy * d.ncx;
    return d;
}

long long ckpt_coarse_size(int nz, int ny, int nx) {
    return (long long)((nz + 1) / 2) * ((ny + 1) / 2) * ((nx + 1) / 2);
}

template <typename T>
cudaError_t launch_ckpt_encode(const T *u, const T *sub, int ns, int nz, int ny, int nx, int px,
                               long long sst, int kind, unsigned *bits, uint16_t *fine,
                               uint16_t *coarse, float *fscale, float *cscale, cudaStream_t st) {
    const CkDims d = ck_dims(nz, ny, nx, px, sst);
    const bool scaled = kind == ESI_CKPT_F16;
    if (px % CK_CH != 0) return cudaErrorInvalidValue;
    const dim3 gc(std::min(d.ncz * d.ncy, 2048), ns),
        gf(blocks_for((long long)nz * ny * (px / CK_CH), 4096), ns);
    if (scaled) {
        cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned) * 2 * ns, st);
        if (e != cudaSuccess) return e;
        ck_coarse_kernel<T><<<gc, RT, 0, st>>>(u, sub, d, 0, kind, bits, coarse, cscale);
    }
    ck_coarse_kernel<T><<<gc, RT, 0, st>>>(u, sub, d, 1, kind, bits, coarse, cscale);
    if (scaled)
        ck_fine_kernel<T><<<gf, RT, 0, st>>>(u, sub, d, 0, kind, bits + ns, coarse, cscale, fine,
                                             fscale);
    ck_fine_kernel<T><<<gf, RT, 0, st>>>(u, sub, d, 1, kind, bits + ns, coarse, cscale, fine,
                                         fscale);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ckpt_decode(const uint16_t *fine, const uint16_t *coarse, const float *fscale,
                               const float *cscale, int ns, int nz, int ny, int nx, int px,
                               long long sst, int kind, const T *base, T *u, cudaStream_t st) {
    const CkDims d = ck_dims(nz, ny, nx, px, sst);
    if (px % CK_CH != 0) return cudaErrorInvalidValue;
    ck_decode_kernel<T><<<dim3(blocks_for((long long)nz * ny * (px / CK_CH), 4096), ns), RT, 0,
                          st>>>(fine, coarse, fscale, cscale, d, kind, base, u);
    return cudaGetLastError();
}

namespace {

// Blocked DTFT (Eq. "dtft"): acc[s][m][cell] += sum_k snap[k][s][cell] e^{+j 2 pi f_m t_k} for
// the K <= DFT_BLOCK_MAX states of one block, twid[k][m] = (cos, sin) of their phases.  A thread
// takes 16 bytes of cells (pads included: they hold zeros, chunks wholly in the pad are
// skipped) and M frequencies in registers, so the K stash planes are read once for up to
// M = 8 frequencies; the block's twiddles of those frequencies are staged in shared memory,
// and the states are loaded four at a time ahead of their sums (accumulated in step order).
// The grid holds as many blocks as are resident at once and strides over the cells.
constexpr int DFT_MCH = 8;

template <typename T, int M>
__global__ void __launch_bounds__(RT) dft_block_kernel(const T *snap, int K, int ns, long long sst,
                                                       int nx, int px, int nf, const T *twid,
                                                       T *acc) {
    constexpr int VEC = V16<T>::n;
    __shared__ T tw[DFT_BLOCK_MAX][M][2];
    const int s = blockIdx.y;
    const long long nch = sst / VEC;
    const T *sn0 = snap + (long long)s * sst;
    const long long kst = (long long)ns * sst;   // stash slot stride
    for (int m0 = 0; m0 < nf; m0 += M) {
        __syncthreads();   // the previous chunk's twiddles are no longer read
        for (int t = threadIdx.x; t < K * M; t += RT) {
            const int k = t / M, j = t - k * M;
            const bool in = m0 + j < nf;
            tw[k][j][0] = in ? twid[((long long)k * nf + m0 + j) * 2] : T(0);
            tw[k][j][1] = in ? twid[((long long)k * nf + m0 + j) * 2 + 1] : T(0);
        }
        __syncthreads();
        const int mn = min(M, nf - m0);
        for (long long c = (long long)blockIdx.x * RT + threadIdx.x; c < nch;
             c += (long long)gridDim.x * RT) {
            const long long cell = c * VEC;
            if ((int)(cell % px) >= nx) continue;   // a chunk of pad cells only: never written
            T re[M][VEC], im[M][VEC];
#pragma unroll
            for (int j = 0; j < M; ++j)
#pragma unroll
                for (int i = 0; i < VEC; ++i) re[j][i] = im[j][i] = T(0);
            const T *src = sn0 + cell;
            int k = 0;
            for (; k + 4 <= K; k += 4) {
                V16<T> u[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    u[q] = *reinterpret_cast<const V16<T> *>(src + (long long)(k + q) * kst);
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int j = 0; j < M; ++j) {
                        const T cs = tw[k + q][j][0], sn = tw[k + q][j][1];
#pragma unroll
                        for (int i = 0; i < VEC; ++i) {
                            re[j][i] += u[q].v[i] * cs;
                            im[j][i] += u[q].v[i] * sn;
                        }
                    }
            }
            for (; k < K; ++k) {
                const V16<T> u = *reinterpret_cast<const V16<T> *>(src + (long long)k * kst);
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const T cs = tw[k][j][0], sn = tw[k][j][1];
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        re[j][i] += u.v[i] * cs;
                        im[j][i] += u.v[i] * sn;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < M; ++j) {
                if (j >= mn) break;
                // VEC complex values = 32 bytes = two 16-byte vectors
                V16<T> *a = reinterpret_cast<V16<T> *>(acc + (((long long)s * nf + m0 + j) * sst + cell) * 2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    V16<T> av = a[h];
#pragma unroll
                    for (int i = 0; i < VEC / 2; ++i) {
                        av.v[2 * i] += re[j][h * VEC / 2 + i];
                        av.v[2 * i + 1] += im[j][h * VEC / 2 + i];
                    }
                    a[h] = av;
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RT) idft_block_kernel(const T *qb, int K, int kst, int ns,
                                                        long long sst, int nf, const T *tw, T *src) {
    constexpr int VEC = V16<T>::n;
    __shared__ T tws[DFT_BLOCK_MAX * FD_MAXF * 2];   // the block's twiddles, staged once
    for (int t = threadIdx.x; t < K * nf * 2; t += RT) tws[t] = tw[t];
    __syncthreads();
    const int s = blockIdx.y;
    const long long nch = sst / VEC;
    for (long long c = (long long)blockIdx.x * RT + threadIdx.x; c < nch;
         c += (long long)gridDim.x * RT) {
        const long long cell = c * VEC;
        T a[FD_MAXF][VEC], b[FD_MAXF][VEC];
#pragma unroll
        for (int m = 0; m < FD_MAXF; ++m) {
            if (m >= nf) break;
            const V16<T> *q = reinterpret_cast<const V16<T> *>(qb + (((long long)s * nf + m) * sst + cell) * 2);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const V16<T> v = q[h];
#pragma unroll
                for (int i = 0; i < VEC / 2; ++i) {
                    a[m][h * VEC / 2 + i] = v.v[2 * i];
                    b[m][h * VEC / 2 + i] = v.v[2 * i + 1];
                }
            }
        }
        for (int k = 0; k < K; ++k) {
            V16<T> o;
#pragma unroll
            for (int i = 0; i < VEC; ++i) o.v[i] = T(0);
#pragma unroll
            for (int m = 0; m < FD_MAXF; ++m) {
                if (m >= nf) break;
                const T C = tws[(k * nf + m) * 2], D = tws[(k * nf + m) * 2 + 1];
#pragma unroll
                for (int i = 0; i < VEC; ++i) o.v[i] += a[m][i] * C + b[m][i] * D;
            }
            *reinterpret_cast<V16<T> *>(src + ((long long)s * kst + k) * sst + cell) = o;
        }
    }
}

// out_m += pb2 sum_m' G[m][m'] p_m' (the lambda B^2 term of Eq. "normaldtft": B commutes with
// F, so F lambda B^2 F^H / nt = lambda B^2 G), with the partials of Re <p, out>
template <typename T>
__global__ void fd_b2g_dot_kernel(T *out, const T *p, const T *pb2, const double *G, int nf,
                                  long long sst, const int *active, double *part) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    double acc = 0.0;
    for (long long c = (long long)blockIdx.x * RT + threadIdx.x; c < sst;
         c += (long long)gridDim.x * RT) {
        const T w = pb2[(long long)s * sst + c];
        T pr[FD_MAXF], pi[FD_MAXF];
#pragma unroll
        for (int m = 0; m < FD_MAXF; ++m) {
            if (m >= nf) break;
            const long long o = (((long long)s * nf + m) * sst + c) * 2;
            pr[m] = p[o];
            pi[m] = p[o + 1];
        }
#pragma unroll
        for (int m = 0; m < FD_MAXF; ++m) {
            if (m >= nf) break;
            T gr = T(0), gi = T(0);
#pragma unroll
            for (int k = 0; k < FD_MAXF; ++k) {
                if (k >= nf) break;
                const T Gr = T(G[(m * nf + k) * 2]), Gi = T(G[(m * nf + k) * 2 + 1]);
                gr += Gr * pr[k] - Gi * pi[k];
                gi += Gr * pi[k] + Gi * pr[k];
            }
            const long long o = (((long long)s * nf + m) * sst + c) * 2;
            const T orr = out[o] + w * gr, oi = out[o + 1] + w * gi;
            out[o] = orr;
            out[o + 1] = oi;
            acc += double(pr[m]) * double(orr) + double(pi[m]) * double(oi);
        }
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
}

// z = w r per cell at every frequency (w = 1 / (lambda B^2)), with the partials of Re <r, z>:
// the diagonal preconditioner of the frequency-domain CG
template <typename T>
__global__ void fd_precond_kernel(T *z, const T *r, const T *w, int nf, long long sst,
                                  const int *active, double *part) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    double acc = 0.0;
    for (long long c = (long long)blockIdx.x * RT + threadIdx.x; c < sst;
         c += (long long)gridDim.x * RT) {
        const T wc = w[(long long)s * sst + c];
        for (int m = 0; m < nf; ++m) {
            const long long o = (((long long)s * nf + m) * sst + c) * 2;
            const T r0 = r[o], r1 = r[o + 1];
            const T z0 = wc * r0, z1 = wc * r1;
            z[o] = z0;
            z[o + 1] = z1;
            acc += double(r0) * double(z0) + double(r1) * double(z1);
        }
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = t;
}

}  // namespace

template <typename T>
cudaError_t launch_fd_precond(T *z, const T *r, const T *w, int nf, int ns, long long sst,
                              const int *active, double *part, cudaStream_t st) {
    fd_precond_kernel<T><<<dim3(DVEC_NBLK, ns), RT, 0, st>>>(z, r, w, nf, sst, active, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_idft_block(const T *qb, int K, int kst, int ns, long long sst, int nf,
                              const T *tw, T *src, cudaStream_t st) {
    if (nf < 1 || nf > FD_MAXF || K < 1 || K > kst || K > DFT_BLOCK_MAX) return cudaErrorInvalidValue;
    // the resident blocks, shared among the shots (grid-stride over the cells)
    static PerDevice slots;
    int nres = 0;
    if (per_device(slots, &nres, [](int *out) {
            int dev = 0, nsm = 0, nb = 0;
            cudaError_t r;
            if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
            if ((r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
                return r;
            if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, idft_block_kernel<T>, RT, 0)) !=
                cudaSuccess)
                return r;
            *out = std::max(1, nb) * std::max(1, nsm);
            return cudaSuccess;
        }) != cudaSuccess)
        nres = 1024;
    const int per_shot = std::max(1, nres / std::max(1, ns));
    idft_block_kernel<T><<<dim3(blocks_for(sst / V16<T>::n, per_shot), ns), RT, 0, st>>>(
        qb, K, kst, ns, sst, nf, tw, src);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fd_b2g_dot(T *out, const T *p, const T *pb2, const double *G, int nf, int ns,
                              long long sst, const int *active, double *part, cudaStream_t st) {
    if (nf > FD_MAXF) return cudaErrorInvalidValue;
    fd_b2g_dot_kernel<T><<<dim3(DVEC_NBLK, ns), RT, 0, st>>>(out, p, pb2, G, nf, sst, active, part);
    return cudaGetLastError();
}

namespace {
// resident blocks of one fold instantiation on the current device (SMs x blocks per SM)
template <typename T, int M>
int dft_block_slots() {
    static PerDevice slots;
    int v = 0;
    cudaError_t e = per_device(slots, &v, [](int *out) {
        int dev = 0, nsm = 0, nb = 0;
        cudaError_t r;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
        if ((r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return r;
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dft_block_kernel<T, M>, RT, 0)) !=
            cudaSuccess)
            return r;
        *out = std::max(1, nb) * std::max(1, nsm);
        return cudaSuccess;
    });
    return e == cudaSuccess ? v : 1024;
}

template <typename T, int M>
cudaError_t go_dft_block(const T *snap, int K, int ns, long long sst, int nx, int px, int nf,
                         const T *twid, T *acc, cudaStream_t st) {
    // the resident blocks, shared among the shots
    const int per_shot = std::max(1, dft_block_slots<T, M>() / std::max(1, ns));
    dft_block_kernel<T, M><<<dim3(blocks_for(sst / V16<T>::n, per_shot), ns), RT, 0, st>>>(
        snap, K, ns, sst, nx, px, nf, twid, acc);
    return cudaGetLastError();
}
}  // namespace

// The longest block (DFT_BLOCK_MAX, 32 or DFT_BLOCK steps) whose stash, steps x the bytes of
// one stashed state of every shot, takes at most 1/16 of the device's memory: the
// accumulators are read and written once per block, the stash twice per step.
int dft_block_steps(long long stash_plane_bytes, size_t device_bytes) {
    int k = DFT_BLOCK_MAX;
    while (k > DFT_BLOCK && (double)k * (double)stash_plane_bytes > (double)device_bytes / 16.0) k /= 2;
    return k;
}

template <typename T>
cudaError_t launch_dft_block(const T *snap, int K, int ns, long long sst, int nx, int px, int nf,
                             const T *twid, T *acc, cudaStream_t st) {
    if (K < 1 || K > DFT_BLOCK_MAX || nf < 1) return cudaErrorInvalidValue;
    switch (std::min(nf, DFT_MCH)) {
        case 1: return go_dft_block<T, 1>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 2: return go_dft_block<T, 2>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 3: return go_dft_block<T, 3>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 4: return go_dft_block<T, 4>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 5: return go_dft_block<T, 5>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 6: return go_dft_block<T, 6>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        case 7: return go_dft_block<T, 7>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
        default: return go_dft_block<T, 8>(snap, K, ns, sst, nx, px, nf, twid, acc, st);
    }
}

// out[i] = sum_g parts[g][i], g in order (the shot groups' partial gradients)
template <typename T>
__global__ void sum_parts_kernel(T *out, const T *parts, int G, long long n) {
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n; i += (long long)gridDim.x * RT) {
        T v = parts[i];
        for (int g = 1; g < G; ++g) v += parts[(long long)g * n + i];
        out[i] = v;
    }
}

template <typename T>
cudaError_t launch_sum_parts(T *out, const T *parts, int G, long long n, cudaStream_t st) {
    sum_parts_kernel<T><<<blocks_for(n, 2048), RT, 0, st>>>(out, parts, G, n);
    return cudaGetLastError();
}
template cudaError_t launch_sum_parts<float>(float *, const float *, int, long long, cudaStream_t);
template cudaError_t launch_sum_parts<double>(double *, const double *, int, long long, cudaStream_t);

template <typename T>
cudaError_t launch_dft_output(const T *acc, long long sst, int rows, int nx, int px, int ns,
                              int nf, int half, void *out, unsigned *bits, float *scales_dev,
                              cudaStream_t st) {
    const long long N = (long long)rows * nx;
    if (half) {
        cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned) * ns * nf, st);
        if (e != cudaSuccess) return e;
        dft_absmax_kernel<T><<<dim3(blocks_for(2 * sst, 1024), ns * nf), RT, 0, st>>>(acc, sst, bits);
    }
    dft_out_kernel<T><<<dim3(blocks_for(N, 1024), ns * nf), RT, 0, st>>>(acc, sst, rows, nx, px,
                                                                        half, bits, out, scales_dev);
    return cudaGetLastError();
}

namespace {

// The penalty of Eq. "esi" (WRI: "wrimisfit"): per-shot partials of 1/2 sum pb2 q^2 over the
// caller's dense space-time field q[s][t][rows][nx], pb2 = beta B^2 pitched per shot.  A block
// walks (t, row) lines; its threads stride along x.
template <typename T>
__global__ void penalty_kernel(const T *q, const T *pb2, int nt, long long rows, int nx, int px,
                               long long sst, double *part) {
    const int s = blockIdx.y;
    const long long nlines = (long long)nt * rows;
    const T *qs = q + (long long)s * nlines * nx;
    double acc = 0.0;
    for (long long l = blockIdx.x; l < nlines; l += gridDim.x) {
        const T *ql = qs + l * nx;
        const T *wl = pb2 + (long long)s * sst + (l % rows) * px;
        for (int x = threadIdx.x; x < nx; x += RT) {
            const T v = ql[x];
            acc += double(wl[x] * v * v);
        }
    }
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = 0.5 * t;
}

// Model-space vectors of the outer loop (dense, any length): <a, b> and max |a| partials in
// double, and z = alpha x + beta y, clamped to [lo, hi] when lo < hi.
template <typename T>
__global__ void mdot_kernel(const T *a, const T *b, long long n, double *part) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n;
         i += (long long)gridDim.x * RT)
        acc += double(a[i]) * double(b[i]);
    const double t = block_sum_d(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <typename T>
__global__ void mamax_kernel(const T *a, long long n, double *part) {
    __shared__ double red[RT / 32];
    double m = 0.0;
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n;
         i += (long long)gridDim.x * RT)
        m = fmax(m, fabs(double(a[i])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RT / 32; ++w) t = fmax(t, red[w]);
        part[blockIdx.x] = t;
    }
}

template <typename T>
__global__ void mlincomb_kernel(T *z, double alpha, const T *x, double beta, const T *y,
                                long long n, double lo, double hi) {
    for (long long i = (long long)blockIdx.x * RT + threadIdx.x; i < n;
         i += (long long)gridDim.x * RT) {
        double v = alpha * double(x[i]);
        if (y) v += beta * double(y[i]);
        if (lo < hi) v = fmin(fmax(v, lo), hi);
        z[i] = T(v);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_penalty(const T *q, const T *pb2, int ns, int nt, long long rows, int nx,
                           int px, long long sst, double *part, int nblk, cudaStream_t st) {
    penalty_kernel<T><<<dim3(nblk, ns), RT, 0, st>>>(q, pb2, nt, rows, nx, px, sst, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mdot(const T *a, const T *b, long long n, double *part, int nblk,
                        cudaStream_t st) {
    mdot_kernel<T><<<nblk, RT, 0, st>>>(a, b, n, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mamax(const T *a, long long n, double *part, int nblk, cudaStream_t st) {
    mamax_kernel<T><<<nblk, RT, 0, st>>>(a, n, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mlincomb(T *z, double alpha, const T *x, double beta, const T *y, long long n,
                            double lo, double hi, cudaStream_t st) {
    mlincomb_kernel<T><<<blocks_for(n, 2048), RT, 0, st>>>(z, alpha, x, beta, y, n, lo, hi);
    return cudaGetLastError();
}

#define ESI_INST(T)                                                                              \
    template cudaError_t launch_setup_cc<T>(const T *, T *, int, int, int, int, double, double,  \
                                            double *, int, cudaStream_t);                        \
    template cudaError_t launch_dot<T>(const T *, const T *, long long, long long, int, double *, \
                                       int, const int *, cudaStream_t);                          \
    template cudaError_t launch_cg_update<T>(T *, T *, const T *, const T *, long long, int, int, \
                                             int, const double *, const int *, double *,         \
                                             double *, int, const T *, long long, int,           \
                                             cudaStream_t);                                      \
    template cudaError_t launch_b2_maps<T>(T *, T *, int, int, int, int, int, T, T, T,           \
                                           const double *, int, cudaStream_t);                   \
    template cudaError_t launch_sub_from<T>(T *, const T *, long long, cudaStream_t);            \
    template cudaError_t launch_dvec_ident_dot<T>(T *, const T *, const long long *, const int *, \
                                                  double *, int, cudaStream_t);                  \
    template cudaError_t launch_dvec_update<T>(T *, T *, const T *, const T *, const long long *, \
                                               const double *, const int *, double *, int,       \
                                               cudaStream_t);                                    \
    template cudaError_t launch_dvec_xpby<T>(T *, const T *, const long long *, const double *,   \
                                             const int *, int, cudaStream_t);                    \
    template cudaError_t launch_scale_to_dense<T>(T *, const T *, const T *, int, int, int, int,  \
                                                  int, long long, cudaStream_t);                 \
    template cudaError_t launch_add_b2p<T>(T *, const T *, int, int, int, int, int, T, T, T,     \
                                           const double *, cudaStream_t);                        \
    template cudaError_t launch_residual<T>(T *, const T *, long long, double *, int,            \
                                            cudaStream_t);                                       \
    template cudaError_t launch_grad_finalize<T>(const T *, int, long long, const T *, int, int, \
                                                 int, int, double, double, double, int, T *,     \
                                                 cudaStream_t);                                  \
    template cudaError_t launch_ckpt_encode<T>(const T *, const T *, int, int, int, int, int,    \
                                               long long, int, unsigned *, uint16_t *,           \
                                               uint16_t *, float *, float *, cudaStream_t);      \
    template cudaError_t launch_ckpt_decode<T>(const uint16_t *, const uint16_t *,              \
                                               const float *, const float *, int, int, int, int, \
                                               int, long long, int, const T *, T *,              \
                                               cudaStream_t);                                    \
    template cudaError_t launch_dft_output<T>(const T *, long long, int, int, int, int, int, int, \
                                              void *, unsigned *, float *, cudaStream_t);       \
    template cudaError_t launch_penalty<T>(const T *, const T *, int, int, long long, int, int,    \
                                           long long, double *, int, cudaStream_t);              \
    template cudaError_t launch_mdot<T>(const T *, const T *, long long, double *, int,           \
                                        cudaStream_t);                                           \
    template cudaError_t launch_mamax<T>(const T *, long long, double *, int, cudaStream_t);      \
    template cudaError_t launch_mlincomb<T>(T *, double, const T *, double, const T *, long long,  \
                                            double, double, cudaStream_t);                       \
    template cudaError_t launch_fd_precond<T>(T *, const T *, const T *, int, int, long long,     \
                                              const int *, double *, cudaStream_t);              \
    template cudaError_t launch_idft_block<T>(const T *, int, int, int, long long, int, const T *, \
                                              T *, cudaStream_t);                                \
    template cudaError_t launch_fd_b2g_dot<T>(T *, const T *, const T *, const double *, int, int, \
                                              long long, const int *, double *, cudaStream_t);   \
    template cudaError_t launch_dft_block<T>(const T *, int, int, long long, int, int, int,      \
                                             const T *, T *, cudaStream_t);

ESI_INST(float)
ESI_INST(double)
#undef ESI_INST

}  // namespace esi
