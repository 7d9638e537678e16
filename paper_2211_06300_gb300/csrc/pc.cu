// Learned CG preconditioner: a 4-level U-Net with 32 channels on time-grouped images.
//
// Applied to the CG residual r of one shot: s = r / (beta B^2) (the diagonal
// preconditioner), pack() groups G = 16 consecutive time samples as channels and averages
// 2 x 2 cells, the network maps these images to a coarse correction y, and
//     z = s + up2(y)
// is the preconditioned residual (the paper's conclusion asks for a preconditioner that
// cuts the inner CG iterations; the network is trained on CG residual / error pairs).
//
// Activations are BF16, channels-last [img][h][w][c].  Every 3 x 3 convolution is an
// implicit GEMM on the 5th-generation tensor cores: a tile is 128 output pixels of one row
// (M = 128), N = output channels, and each of the 9 taps contributes K = input channels.
// The 3-row input patch of a tile is staged by TMA (one box per 8-channel chunk, zero fill
// at the image edges) in the canonical no-swizzle K-major layout, so every tap is the same
// patch seen through a shared-memory descriptor shifted by (dy * 130 + dx) * 16 bytes.  One
// thread issues tcgen05.mma into a TMEM accumulator; the four warps read it back with
// tcgen05.ld for the bias / ReLU / BF16 epilogue.  Training reuses the same kernel for the
// input gradient (flipped, transposed weights); the weight gradient, whose M is only 16 or
// 32 channels (below the tcgen05 minimum of 64 rows), runs on warp-level mma.sync.
#include <cuda_bf16.h>

#include <algorithm>

#include "esi_internal.h"
#include "esi_pc.h"

namespace esi {
namespace pcnet {
namespace {

constexpr int TM = 128;              // output pixels per conv tile
constexpr int PW = TM + 2;           // patch width (1-pixel halo each side)
constexpr int NTH = 128;             // conv block: 4 warps
constexpr long long WAIT_LIMIT = 1ll << 26;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned phase) {
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *tm, int c, int x, int y,
                                            int n, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c), "r"(x), "r"(y), "r"(n),
        "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): start, leading-dimension byte offset (between
// core matrices along K), stride byte offset (between 8-row groups along M/N), no swizzle.
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version of the 5th-generation tensor cores
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) |
           ((unsigned)(M >> 4) << 24);
}

template <int N>
__device__ __forceinline__ void tmem_ld(unsigned taddr, float *v);

template <>
__device__ __forceinline__ void tmem_ld<16>(unsigned taddr, float *v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_ld<32>(unsigned taddr, float *v) {
    tmem_ld<16>(taddr, v);
    tmem_ld<16>(taddr + 16, v + 16);
}

template <typename OUT>
__device__ __forceinline__ void store_row(OUT *dst, const float *v, int n);

template <>
__device__ __forceinline__ void store_row<__nv_bfloat16>(__nv_bfloat16 *dst, const float *v, int n) {
    for (int c = 0; c < n; c += 8) {
        uint4 q;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[c + 2 * i], v[c + 2 * i + 1]);
        *reinterpret_cast<uint4 *>(dst + c) = q;
    }
}

template <>
__device__ __forceinline__ void store_row<float>(float *dst, const float *v, int n) {
    for (int c = 0; c < n; c += 4)
        *reinterpret_cast<float4 *>(dst + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
}

// y[img][h][w][co] = act(b[co] + sum_taps sum_ci x[img][h+dy-1][w+dx-1][ci] W[tap][ci][co])
// wprep: [9][CIN/8][COUT][8] BF16 (the canonical K-major B operand per tap).
//
// A CTA owns a strip (one image, 128 columns, all H rows) at a time and marches down it: input
// rows arrive by TMA in a ring of RROWS slots (each row once per strip), so output row y
// takes its three taps' rows from slots y - 1, y, y + 1.  One thread waits for the rows,
// issues the 9 x CIN/16 MMAs of row y into one of two TMEM accumulators and commits; the
// four warps meanwhile drain row y - 1 from the other accumulator (bias, ReLU, scale,
// store).  When row y - 1's MMAs are complete its oldest input slot is refilled, RROWS - 3
// rows ahead of use.  Every wait is bounded; on a timeout the CTA records the error, lets
// its copies and MMAs in flight finish and leaves.
constexpr int RROWS = 6;

template <int CIN, int COUT>
struct ConvGeom {
    static constexpr int NCH = CIN / 8;
    static constexpr int RB = (PW * 16 + 127) / 128 * 128;   // one 8-channel row chunk (2176 B)
    static constexpr int SLOT = NCH * RB;                      // one staged input row
    static constexpr int RING = RROWS * SLOT;
    static constexpr int WTAP = CIN * COUT * 2;                // one tap's weights
    static constexpr int SMEM = (RING + 1023) / 1024 * 1024 + 9 * WTAP + 1024;
    static constexpr int TCOLS = 2 * COUT <= 32 ? 32 : (2 * COUT <= 64 ? 64 : 128);
};

template <int CIN, int COUT, bool RELU, typename OUT>
__global__ void __launch_bounds__(NTH) conv3x3_tc_kernel(const __grid_constant__ CUtensorMap in_map,
                                                         const __nv_bfloat16 *__restrict__ wprep,
                                                         const float *__restrict__ bias,
                                                         OUT *__restrict__ out, int nimg, int H,
                                                         int W, int *dev_err, ConvEpi epi) {
    using Gm = ConvGeom<CIN, COUT>;
    constexpr int NCH = Gm::NCH, RB = Gm::RB, SLOT = Gm::SLOT;
    constexpr unsigned IDESC = idesc_bf16(TM, COUT);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align the dynamic shared memory base at run time (TMA destinations need 128 bytes)
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *ring = smem;
    unsigned char *wsm = smem + (Gm::RING + 1023) / 1024 * 1024;
    __shared__ __align__(8) unsigned long long bar_full[RROWS], bar_mma[2];
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int i = tid; i < 9 * Gm::WTAP / 16; i += NTH)
        reinterpret_cast<uint4 *>(wsm)[i] = reinterpret_cast<const uint4 *>(wprep)[i];
    if (tid == 0) {
        for (int k = 0; k < RROWS; ++k) mbar_init(&bar_full[k]);
        mbar_init(&bar_mma[0]);
        mbar_init(&bar_mma[1]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the weights were written through the generic proxy; the tensor core reads them
    // through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "n"(Gm::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    const int tiles_x = (W + TM - 1) / TM;
    const long long nstrips = (long long)nimg * tiles_x;
    const int nin = H + 2;            // input rows -1 .. H of a strip
    unsigned seq_in = 0;              // input rows staged by this CTA before the current strip
    unsigned seq_out = 0;             // output rows computed before the current strip
    int issued = 0;                   // input rows of the current strip issued so far
    int mma_open = -1;                // output row whose MMAs may still be in flight
    bool late = false;
    // input row j of the strip: slot (seq_in + j) % RROWS, completed phase parity
    auto slot_of = [&](int j) { return (seq_in + (unsigned)j) % RROWS; };
    auto par_in = [&](int j) { return ((seq_in + (unsigned)j) / RROWS) & 1u; };
    for (long long st = blockIdx.x; st < nstrips; st += gridDim.x) {
        const int tx = int(st % tiles_x), img = int(st / tiles_x);
        const int x0 = tx * TM;
        auto issue = [&](int j) {   // thread 0: stage input row j - 1
            const unsigned k = slot_of(j);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                             smem_u32(&bar_full[k])),
                         "r"((unsigned)(NCH * PW * 16))
                         : "memory");
#pragma unroll
            for (int c = 0; c < NCH; ++c)
                tma_load_4d(ring + k * SLOT + c * RB, &in_map, 8 * c, x0 - 1, j - 1, img,
                            &bar_full[k]);
        };
        issued = min(nin, RROWS);
        if (tid == 0)
            for (int j = 0; j < issued; ++j) issue(j);
        const float sc = epi.oscale ? epi.oscale[img] : 1.0f;   // per-image output factor
        float isc = 1.0f;                                        // per-image input factor
        if (epi.irms) {
            const float r = epi.irms[img];
            isc = r > 0.0f ? 1.0f / r : 0.0f;
        }
        auto epilogue = [&](int y, unsigned o) {
            float v[COUT];
            tmem_ld<COUT>(tmem + ((unsigned)(warp * 32) << 16) + (o & 1u) * COUT, v);
            const int px = x0 + warp * 32 + lane;
            if (px < W) {
#pragma unroll
                for (int c = 0; c < COUT; ++c) {
                    float a = v[c] * isc + (bias ? bias[c] : 0.0f);
                    v[c] = sc * (RELU ? fmaxf(a, 0.0f) : a);
                }
                if (epi.nchw) {   // planes [img][c][H][W]: coalesced along px per channel
                    OUT *o0 = out + ((long long)img * COUT * H + y) * W + px;
#pragma unroll
                    for (int c = 0; c < COUT; ++c) o0[(long long)c * H * W] = OUT(v[c]);
                } else {
                    store_row<OUT>(out + (((long long)img * H + y) * W + px) * COUT, v, COUT);
                }
            }
        };
        for (int y = 0; y < H; ++y) {
            const unsigned o = seq_out + (unsigned)y;
            if (tid == 0) {
                bool ok = true;
#pragma unroll
                for (int d = 0; d < 3; ++d) ok &= mbar_wait(&bar_full[slot_of(y + d)], par_in(y + d));
                late |= !ok;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned wb = smem_u32(wsm), acc_addr = tmem + (o & 1u) * COUT;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const unsigned pa = smem_u32(ring + slot_of(y + dy) * SLOT);
#pragma unroll
                    for (int ks = 0; ks < CIN / 16; ++ks) {
                        const unsigned long long da = sdesc(pa + ks * 2 * RB + dx * 16, RB, 128);
                        const unsigned long long db =
                            sdesc(wb + tap * Gm::WTAP + ks * 2 * COUT * 16, COUT * 16, 128);
                        const unsigned acc = (tap | ks) ? 1u : 0u;
                        asm volatile(
                            "{ .reg .pred p; setp.ne.u32 p, %4, 0;"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
                                acc_addr),
                            "l"(da), "l"(db), "r"(IDESC), "r"(acc)
                            : "memory");
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&bar_mma[o & 1u]))
                    : "memory");
            }
            mma_open = y;
            if (y >= 1) {
                // row y - 1: its MMAs are complete once its commit arrives
                late |= !mbar_wait(&bar_mma[(o - 1) & 1u], ((o - 1) >> 1) & 1u);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                epilogue(y - 1, o - 1);
                // input row y - 2 (sequence j = y - 1) had its last reader in row y - 1
                if (tid == 0)
                    while (issued < nin && issued <= y - 1 + RROWS) issue(issued++);
                else
                    issued = min(nin, max(issued, y + RROWS));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            if (__syncthreads_or(late)) goto timeout;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        {
            const unsigned o = seq_out + (unsigned)(H - 1);
            late |= !mbar_wait(&bar_mma[o & 1u], (o >> 1) & 1u);
            mma_open = -1;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            epilogue(H - 1, o);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(late)) goto timeout;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        seq_in += (unsigned)nin;
        seq_out += (unsigned)H;
    }
    goto done;
timeout:
    // let the copies and the MMAs in flight finish before the TMEM and shared memory go
    if (tid == 0) {
        atomicExch(dev_err, DEV_ERR_TMA_TIMEOUT);
        for (int j = max(0, issued - RROWS); j < issued; ++j) mbar_wait(&bar_full[slot_of(j)], par_in(j));
        if (mma_open >= 0) {
            const unsigned o = seq_out + (unsigned)mma_open;
            mbar_wait(&bar_mma[o & 1u], (o >> 1) & 1u);
        }
    }
    __syncthreads();
done:
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "n"(Gm::TCOLS)
                     : "memory");
}

// ----------------------------------------------------------------------------- weights
// master FP32 W[3][3][cin][cout] -> BF16 [tap][cin/8][cout][8]; with flip, the input-gradient
// weights W'[tap'][co][ci] = W[8 - tap][ci][co] (cin' = cout, cout' = cin)
__global__ void wprep_kernel(const float *W, __nv_bfloat16 *out, int cin, int cout, int flip) {
    const int ci_ = flip ? cout : cin, co_ = flip ? cin : cout;
    const int total = 9 * ci_ * co_;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        // i enumerates the output layout [tap][kc][n][e]
        const int e = i % 8, n = (i / 8) % co_, kc = (i / (8 * co_)) % (ci_ / 8), tap = i / (ci_ * co_);
        const int k = kc * 8 + e;  // input channel of this (possibly flipped) convolution
        float w;
        if (!flip) w = W[(tap * cin + k) * cout + n];
        else w = W[((8 - tap) * cin + n) * cout + k];
        out[i] = __float2bfloat16_rn(w);
    }
}

// ----------------------------------------------------------------------------- data movement
// residual -> network input: img[(s*ng + g)][hc][wc][c] = 1/4 sum_{2x2} r[s][16g+c] * ipb2[s].
// A block takes whole output rows (s, g, zc); its threads run along the row, each producing
// one pixel's 16 channels in two halves of 8 (few live registers, many loads in flight).
__global__ void __launch_bounds__(256, 4) pack_kernel(const float *r, const float *ipb2,
                                                      __nv_bfloat16 *img, int ns, int nt, int ng,
                                                      int nz, int nx, int px, long long sst,
                                                      int hc, int wc, int scale_by_map, int dense) {
    const int nrow = ns * ng * hc;
    const long long plane = dense ? (long long)nz * nx : sst;
    const int rstride = dense ? nx : px;
    for (int rw = blockIdx.x; rw < nrow; rw += gridDim.x) {
        const int zc = rw % hc, ig = rw / hc;
        const int g = ig % ng, s = ig / ng;
        const float *rs = r + (long long)s * nt * plane;
        __nv_bfloat16 *orow = img + ((long long)ig * hc + zc) * wc * G;
        for (int xc = threadIdx.x; xc < wc; xc += blockDim.x) {
            // the 2 x 2 cells: rows iz0, iz0 + 1 (if inside), columns ix0, ix0 + 1 (if inside)
            const int iz0 = 2 * zc, ix0 = 2 * xc;
            const bool row2 = iz0 + 1 < nz, col2 = ix0 + 1 < nx;
            float m[2][2] = {{1.0f, 1.0f}, {1.0f, 1.0f}};
            if (scale_by_map) {
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    if (a == 1 && !row2) break;
                    const float *ib = ipb2 + (long long)s * sst + (long long)(iz0 + a) * px + ix0;
                    m[a][0] = ib[0];
                    m[a][1] = col2 ? ib[1] : 0.0f;
                }
            }
            if (!col2) m[0][1] = m[1][1] = 0.0f;
            if (!row2) m[1][0] = m[1][1] = 0.0f;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[G / 2];
#pragma unroll
                for (int c = 0; c < G / 2; ++c) {
                    const int t = G * g + (G / 2) * h + c;
                    float acc = 0.0f;
                    if (t < nt) {
                        const float *rt = rs + (long long)t * plane + (long long)iz0 * rstride + ix0;
#pragma unroll
                        for (int a = 0; a < 2; ++a) {
                            const float *rr = rt + (long long)a * rstride;
                            const bool in = a == 0 || row2;
                            const float r0 = in ? rr[0] : 0.0f;
                            const float r1 = in && col2 ? rr[1] : 0.0f;
                            acc += r0 * m[a][0] + r1 * m[a][1];
                        }
                    }
                    v[c] = 0.25f * acc;
                }
                store_row<__nv_bfloat16>(orow + (long long)xc * G + (G / 2) * h, v, G / 2);
            }
        }
    }
}

// The same packing for the pitched residual (row stride px, a multiple of 32 floats, pads zero):
// a thread takes two neighbouring output pixels, i.e. 4 input columns, and reads them as one
// 16-byte load per row and time sample; a block walks whole output rows.  Columns past nx read
// the zero pads (4 * ceil(nx / 4) <= px), so no column test is needed.
__global__ void __launch_bounds__(256, 4) pack4_kernel(const float *r, const float *ipb2,
                                                       __nv_bfloat16 *img, int ns, int nt, int ng,
                                                       int nz, int px, long long sst, int hc,
                                                       int wc, int scale_by_map) {
    const int nrow = ns * ng * hc, nqd = (wc + 1) / 2;
    for (int rw = blockIdx.x; rw < nrow; rw += gridDim.x) {
        const int zc = rw % hc, ig = rw / hc;
        const int g = ig % ng, s = ig / ng;
        const float *rs = r + (long long)s * nt * sst;
        __nv_bfloat16 *orow = img + ((long long)ig * hc + zc) * wc * G;
        const int iz0 = 2 * zc;
        const bool row2 = iz0 + 1 < nz;
        for (int qd = threadIdx.x; qd < nqd; qd += blockDim.x) {
            const int ix0 = 4 * qd;
            float4 m[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                m[a] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                if (scale_by_map && (a == 0 || row2))
                    m[a] = *reinterpret_cast<const float4 *>(ipb2 + (long long)s * sst +
                                                             (long long)(iz0 + a) * px + ix0);
            }
            if (!row2) m[1] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const bool pix2 = 2 * qd + 1 < wc;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v0[G / 2], v1[G / 2];
#pragma unroll
                for (int c = 0; c < G / 2; ++c) {
                    const int t = G * g + (G / 2) * h + c;
                    float a0 = 0.0f, a1 = 0.0f;
                    if (t < nt) {
                        const float *rt = rs + (long long)t * sst + (long long)iz0 * px + ix0;
                        const float4 u = *reinterpret_cast<const float4 *>(rt);
                        a0 = u.x * m[0].x + u.y * m[0].y;
                        a1 = u.z * m[0].z + u.w * m[0].w;
                        if (row2) {
                            const float4 w = *reinterpret_cast<const float4 *>(rt + px);
                            a0 += w.x * m[1].x + w.y * m[1].y;
                            a1 += w.z * m[1].z + w.w * m[1].w;
                        }
                    }
                    v0[c] = 0.25f * a0;
                    v1[c] = 0.25f * a1;
                }
                store_row<__nv_bfloat16>(orow + (long long)(2 * qd) * G + (G / 2) * h, v0, G / 2);
                if (pix2)
                    store_row<__nv_bfloat16>(orow + (long long)(2 * qd + 1) * G + (G / 2) * h, v1,
                                             G / 2);
            }
        }
    }
}

// 2 x 2 average pooling (zero fill at odd edges), BF16 channels-last, C = 32
__global__ void pool_kernel(const __nv_bfloat16 *in, __nv_bfloat16 *out, long long n, int H, int W,
                            int Ho, int Wo) {
    const long long total = n * Ho * Wo * (C / 8);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = int(i % (C / 8));
        const long long p = i / (C / 8);
        const int x = int(p % Wo);
        const long long r1 = p / Wo;
        const int y = int(r1 % Ho);
        const long long img = r1 / Ho;
        float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int iy = 2 * y + a, ix = 2 * x + b;
                if (iy >= H || ix >= W) continue;
                const uint4 q = *reinterpret_cast<const uint4 *>(in + ((img * H + iy) * W + ix) * C + ch * 8);
                const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __bfloat1622float2(h[k]);
                    acc[2 * k] += f.x;
                    acc[2 * k + 1] += f.y;
                }
            }
        for (int k = 0; k < 8; ++k) acc[k] *= 0.25f;
        store_row<__nv_bfloat16>(out + p * C + ch * 8, acc, 8);
    }
}

// out[h][w] = coarse[h/2][w/2] + skip[h][w]  (C = 32)
__global__ void upadd_kernel(const __nv_bfloat16 *coarse, const __nv_bfloat16 *skip,
                             __nv_bfloat16 *out, long long n, int H, int W, int Hc, int Wc) {
    const long long total = n * H * W * (C / 8);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = int(i % (C / 8));
        const long long p = i / (C / 8);
        const int x = int(p % W);
        const long long r1 = p / W;
        const int y = int(r1 % H);
        const long long img = r1 / H;
        const uint4 a = *reinterpret_cast<const uint4 *>(coarse + ((img * Hc + y / 2) * Wc + x / 2) * C + ch * 8);
        const uint4 b = *reinterpret_cast<const uint4 *>(skip + p * C + ch * 8);
        const __nv_bfloat162 *ha = reinterpret_cast<const __nv_bfloat162 *>(&a);
        const __nv_bfloat162 *hb = reinterpret_cast<const __nv_bfloat162 *>(&b);
        float o[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 fa = __bfloat1622float2(ha[k]), fb = __bfloat1622float2(hb[k]);
            o[2 * k] = fa.x + fb.x;
            o[2 * k + 1] = fa.y + fb.y;
        }
        store_row<__nv_bfloat16>(out + p * C + ch * 8, o, 8);
    }
}

// per-image root-mean-square of BF16 images [n][per]; rms[img] (FP32)
// per-image sum of squares: blocks (chunk, image), 8 BF16 values per load, FP32 within a
// thread, FP64 across threads and blocks
__global__ void img_sumsq_kernel(const __nv_bfloat16 *x, double *acc, long long per) {
    const int img = blockIdx.y;
    const long long n8 = per / 8;   // per is a multiple of G = 16
    const uint4 *v = reinterpret_cast<const uint4 *>(x + (long long)img * per);
    float s = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n8;
         i += (long long)gridDim.x * blockDim.x) {
        const uint4 q = v[i];
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            s += f.x * f.x + f.y * f.y;
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = double(s);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(acc + img, red[0]);
}

__global__ void img_rms_kernel(const double *acc, float *rms, int n, long long per) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) rms[i] = float(sqrt(acc[i] / double(per)));
}

__global__ void img_scale_kernel(const __nv_bfloat16 *x, const float *rms, __nv_bfloat16 *xn,
                                 long long per, long long total) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float r = rms[i / per];
        xn[i] = __float2bfloat16_rn(r > 0.0f ? __bfloat162float(x[i]) / r : 0.0f);
    }
}

// g[img][...] *= s[img]
__global__ void img_mul_kernel(float *g, const float *s, long long per, long long total) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        g[i] *= s[i / per];
}

// ----------------------------------------------------------------------------- training
// g (FP32) * relu'(act) -> BF16 operand of the backward convolutions (and back into g)
__global__ void mask_kernel(float *g, const __nv_bfloat16 *act, __nv_bfloat16 *gb, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float v = g[i];
        if (act && !(__bfloat162float(act[i]) > 0.0f)) v = 0.0f;
        g[i] = v;
        gb[i] = __float2bfloat16_rn(v);
    }
}

// g_fine[h][w] += 0.25 g_coarse[h/2][w/2]   (pooling backward)
__global__ void pool_bwd_kernel(float *gf, const float *gc, long long n, int H, int W, int Hc,
                                int Wc) {
    const long long total = n * H * W * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long p = i / C;
        const int x = int(p % W);
        const long long r1 = p / W;
        const int y = int(r1 % H);
        const long long img = r1 / H;
        gf[i] += 0.25f * gc[((img * Hc + y / 2) * Wc + x / 2) * C + c];
    }
}

// g_coarse[h][w] = sum of g_fine over the 2 x 2 block (upsampling backward)
__global__ void up_bwd_kernel(const float *gf, float *gc, long long n, int H, int W, int Hc,
                              int Wc) {
    const long long total = n * Hc * Wc * C;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C);
        const long long p = i / C;
        const int x = int(p % Wc);
        const long long r1 = p / Wc;
        const int y = int(r1 % Hc);
        const long long img = r1 / Hc;
        float s = 0.0f;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const int iy = 2 * y + a, ix = 2 * x + b;
                if (iy < H && ix < W) s += gf[((img * H + iy) * W + ix) * C + c];
            }
        gc[i] = s;
    }
}

__device__ __forceinline__ unsigned pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

// Weight gradient of one tap on warp-level tensor cores (mma.sync m16n8k16, BF16 in, FP32
// accumulate): dW[tap][ci][co] = sum_pixels x[pixel shifted by tap][ci] * gy[pixel][co].
// Block = 4 warps over 64-pixel row segments; the partial of each block goes to part[tap][blk].
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) dw_kernel(const __nv_bfloat16 *x, const __nv_bfloat16 *gy,
                                                  float *part, int nimg, int H, int W) {
    constexpr int SEG = 64;
    __shared__ __nv_bfloat16 xs[SEG][CIN];
    __shared__ __nv_bfloat16 gs[SEG][COUT];
    const int tap = blockIdx.y, dy = tap / 3, dx = tap % 3;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    constexpr int MT = CIN / 16, NTL = COUT / 8;
    // warp w owns rows (ci) 16*(w % MT).. and columns a share of the n-tiles
    float acc[MT][NTL][4];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < NTL; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const int segs_x = (W + SEG - 1) / SEG;
    const long long nseg = (long long)nimg * H * segs_x;
    for (long long sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const int sx = int(sg % segs_x);
        const long long r1 = sg / segs_x;
        const int y = int(r1 % H), img = int(r1 / H);
        const int x0 = sx * SEG;
        const int iy = y + dy - 1;
        for (int i = tid; i < SEG * CIN; i += 128) {
            const int p = i / CIN, c = i % CIN;
            const int ix = x0 + p + dx - 1;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (x0 + p < W && iy >= 0 && iy < H && ix >= 0 && ix < W)
                v = x[(((long long)img * H + iy) * W + ix) * CIN + c];
            xs[p][c] = v;
        }
        for (int i = tid; i < SEG * COUT; i += 128) {
            const int p = i / COUT, c = i % COUT;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (x0 + p < W) v = gy[(((long long)img * H + y) * W + x0 + p) * COUT + c];
            gs[p][c] = v;
        }
        __syncthreads();
        // each warp takes 16 of the 64 pixels (K), all M and N tiles
        const int k0 = warp * 16;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int m0 = mt * 16;
            const unsigned a0 = pack_bf16(xs[k0 + 2 * tig][m0 + gid], xs[k0 + 2 * tig + 1][m0 + gid]);
            const unsigned a1 = pack_bf16(xs[k0 + 2 * tig][m0 + gid + 8], xs[k0 + 2 * tig + 1][m0 + gid + 8]);
            const unsigned a2 = pack_bf16(xs[k0 + 2 * tig + 8][m0 + gid], xs[k0 + 2 * tig + 9][m0 + gid]);
            const unsigned a3 = pack_bf16(xs[k0 + 2 * tig + 8][m0 + gid + 8], xs[k0 + 2 * tig + 9][m0 + gid + 8]);
#pragma unroll
            for (int nt_ = 0; nt_ < NTL; ++nt_) {
                const int n0 = nt_ * 8;
                const unsigned b0 = pack_bf16(gs[k0 + 2 * tig][n0 + gid], gs[k0 + 2 * tig + 1][n0 + gid]);
                const unsigned b1 = pack_bf16(gs[k0 + 2 * tig + 8][n0 + gid], gs[k0 + 2 * tig + 9][n0 + gid]);
                float *d = acc[mt][nt_];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
                    "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                    : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                    : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
            }
        }
        __syncthreads();
    }
    // reduce the 4 warps' accumulators in shared memory, then one partial per block
    __shared__ float red[4][CIN][COUT];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt_ = 0; nt_ < NTL; ++nt_) {
            const int m0 = mt * 16, n0 = nt_ * 8;
            red[warp][m0 + gid][n0 + 2 * tig] = acc[mt][nt_][0];
            red[warp][m0 + gid][n0 + 2 * tig + 1] = acc[mt][nt_][1];
            red[warp][m0 + gid + 8][n0 + 2 * tig] = acc[mt][nt_][2];
            red[warp][m0 + gid + 8][n0 + 2 * tig + 1] = acc[mt][nt_][3];
        }
    __syncthreads();
    float *dst = part + ((long long)tap * gridDim.x + blockIdx.x) * CIN * COUT;
    for (int i = tid; i < CIN * COUT; i += 128) {
        const int m = i / COUT, n = i % COUT;
        dst[i] = red[0][m][n] + red[1][m][n] + red[2][m][n] + red[3][m][n];
    }
}

// dW[tap][ci][co] (+ layout of the master weights) = sum of the block partials, fixed order
__global__ void dw_reduce_kernel(const float *part, float *gW, int nblk, int cin, int cout) {
    const int per = cin * cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 9 * per; i += gridDim.x * blockDim.x) {
        const int tap = i / per, r = i % per;
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[((long long)tap * nblk + b) * per + r];
        gW[i] = float(s);
    }
}

// bias gradient: gb[c] = sum over pixels of g (FP32 [pix][C]), one block per channel
__global__ void bias_grad_kernel(const float *g, float *gb, long long npix, int Cn) {
    const int c = blockIdx.x;
    double s = 0.0;
    for (long long p = threadIdx.x; p < npix; p += blockDim.x) s += g[p * Cn + c];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[c] = float(red[0]);
}

// per-image dots of z = in + y with the target e: dots[img] = (<z,e>, <z,z>, <e,e>)
__global__ void cos_dots_kernel(const __nv_bfloat16 *in, const float *y, const __nv_bfloat16 *e,
                                double *dots, long long per) {
    const int img = blockIdx.x;
    double ze = 0, zz = 0, ee = 0;
    for (long long i = threadIdx.x; i < per; i += blockDim.x) {
        const long long k = (long long)img * per + i;
        const double z = double(__bfloat162float(in[k])) + double(y[k]);
        const double t = double(__bfloat162float(e[k]));
        ze += z * t;
        zz += z * z;
        ee += t * t;
    }
    __shared__ double r[3][256];
    r[0][threadIdx.x] = ze;
    r[1][threadIdx.x] = zz;
    r[2][threadIdx.x] = ee;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) r[q][threadIdx.x] += r[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) dots[3 * img + q] = r[q][0];
}

// gradient of mean_img (1 - <z,e>^2 / (|z|^2 |e|^2)) with respect to y (= with respect to z)
__global__ void cos_grad_kernel(const __nv_bfloat16 *in, const float *y, const __nv_bfloat16 *e,
                                const double *dots, float *gy, long long per, int nimg) {
    const long long total = (long long)nimg * per;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int img = int(k / per);
        const double ze = dots[3 * img], zz = dots[3 * img + 1], ee = dots[3 * img + 2];
        const double z = double(__bfloat162float(in[k])) + double(y[k]);
        const double t = double(__bfloat162float(e[k]));
        double g = 0.0;
        if (zz > 0 && ee > 0) g = (-(2.0 * ze / (zz * ee)) * t + (2.0 * ze * ze / (zz * zz * ee)) * z) / nimg;
        gy[k] = float(g);
    }
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}


// per-shot <s, r>, <y, r>, <s, a>, <y, a> for the flexible CG (a = A p of the previous
// iteration, s = r ipb2, y = up2 of the network's coarse correction), into
// part[q][shot][block], q in that order.  A block takes whole rows (t, iz) of one shot, its
// threads 4 cells (16 bytes) of the row each; a thread's running totals are compensated FP32
// sums, the block's FP64.
__global__ void pc_dots_kernel(const float *r, const float *ap, const float *ipb2,
                               const float *y, double *part, int nt, int ng, int nz, int nx,
                               int px, long long sst, int hc, int wc, const int *active) {
    const int s = blockIdx.y, ns = gridDim.y;
    if (active && !active[s]) return;
    const int rows = nt * nz, nq = (nx + 3) / 4;
    // compensated (Kahan) FP32 sums per thread: FP64 arithmetic is scarce on this part
    float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f}, comp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    auto kadd = [&](int q, float v) {
        const float yv = v - comp[q];
        const float t = sum[q] + yv;
        comp[q] = (t - sum[q]) - yv;
        sum[q] = t;
    };
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int t = row / nz, iz = row - t * nz;
        const long long off = ((long long)s * nt + t) * sst + (long long)iz * px;
        const float *rr = r + off;
        const float *aa = ap ? ap + off : nullptr;
        const float *ib = ipb2 + (long long)s * sst + (long long)iz * px;
        // y: time-sample planes [s][ng * G][hc][wc]
        const float *yr = y + (((long long)s * ng * G + t) * hc + iz / 2) * wc;
        for (int c = threadIdx.x; c < nq; c += blockDim.x) {
            const int x = 4 * c;
            const float4 r4 = *reinterpret_cast<const float4 *>(rr + x);
            const float4 b4 = *reinterpret_cast<const float4 *>(ib + x);
            const float4 a4 = aa ? *reinterpret_cast<const float4 *>(aa + x) : make_float4(0, 0, 0, 0);
            const float y0 = yr[2 * c], y1 = x + 2 < nx ? yr[2 * c + 1] : 0.0f;
            const float rv[4] = {r4.x, r4.y, r4.z, r4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            float f[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (x + k >= nx) break;
                const float sv = rv[k] * bv[k], yv = k < 2 ? y0 : y1;
                f[0] += sv * rv[k];
                f[1] += yv * rv[k];
                f[2] += sv * av[k];
                f[3] += yv * av[k];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) kadd(q, f[q]);
        }
    }
    __shared__ double red[4][256];
#pragma unroll
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = double(sum[q]) - double(comp[q]);
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
#pragma unroll
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 4)
        part[((long long)threadIdx.x * ns + s) * gridDim.x + blockIdx.x] = red[threadIdx.x][0];
}

inline int grid_for(long long n, int cap = 4096) {
    long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

// ----------------------------------------------------------------------------- launchers
cudaError_t make_act_map(CUtensorMap *tm, const void *base, int C_, int W, int H, int n) {
    auto enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)C_, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)C_ * 2, (cuuint64_t)W * C_ * 2,
                                   (cuuint64_t)H * W * C_ * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)PW, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides,
                     box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT, bool RELU, typename OUT>
cudaError_t conv_launch(const void *in, const __nv_bfloat16 *wprep, const float *bias, OUT *out,
                        int nimg, int H, int W, int *dev_err, int nsm, cudaStream_t st,
                        const ConvEpi &epi) {
    using Gm = ConvGeom<CIN, COUT>;
    CUtensorMap tm;
    cudaError_t e = make_act_map(&tm, in, CIN, W, H, nimg);
    if (e != cudaSuccess) return e;
    auto kern = conv3x3_tc_kernel<CIN, COUT, RELU, OUT>;
    static PerDevice cache;
    int per_sm = 0;
    e = per_device(cache, &per_sm, [kern](int *v) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Gm::SMEM);
        if (r != cudaSuccess) return r;
        r = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (r != cudaSuccess) return r;
        // resident CTAs per SM from the shared memory, register and TMEM budgets (a CTA
        // beyond them only waits for its turn: strips are independent)
        int dev = 0, smem_sm = 0, rsv = 0, regs_sm = 0;
        cudaFuncAttributes fa;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess ||
            (r = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
            (r = cudaDeviceGetAttribute(&rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
            (r = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
            (r = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess)
            return r;
        const int by_smem = smem_sm / (Gm::SMEM + (int)fa.sharedSizeBytes + rsv);
        const int by_regs = regs_sm / (NTH * std::max(fa.numRegs, 1));
        *v = std::max(1, std::min({by_smem, by_regs, 512 / Gm::TCOLS}));
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    const long long strips = (long long)nimg * ((W + TM - 1) / TM);
    const int grid = (int)std::min<long long>(strips, (long long)nsm * per_sm);
    kern<<<grid, NTH, Gm::SMEM, st>>>(tm, wprep, bias, out, nimg, H, W, dev_err, epi);
    return cudaGetLastError();
}

#define CONV_INST(CI, CO, R, O)                                                                 \
    template cudaError_t conv_launch<CI, CO, R, O>(const void *, const __nv_bfloat16 *,        \
                                                   const float *, O *, int, int, int, int *,   \
                                                   int, cudaStream_t, const ConvEpi &);
CONV_INST(16, 32, true, __nv_bfloat16)
CONV_INST(32, 32, true, __nv_bfloat16)
CONV_INST(32, 16, false, float)
CONV_INST(16, 32, false, float)
CONV_INST(32, 32, false, float)
#undef CONV_INST

cudaError_t normalize_launch(const __nv_bfloat16 *x, float *rms, double *acc, __nv_bfloat16 *xn,
                             int n, long long per, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * n, st);
    if (e != cudaSuccess) return e;
    const int chunks = (int)std::max<long long>(1, std::min<long long>(32, per / 8 / 256 / 4));
    img_sumsq_kernel<<<dim3(chunks, n), 256, 0, st>>>(x, acc, per);
    img_rms_kernel<<<(n + 255) / 256, 256, 0, st>>>(acc, rms, n, per);
    e = cudaGetLastError();
    if (e != cudaSuccess || !xn) return e;
    img_scale_kernel<<<grid_for((long long)n * per), 256, 0, st>>>(x, rms, xn, per, (long long)n * per);
    return cudaGetLastError();
}

cudaError_t img_mul_launch(float *g, const float *s, int n, long long per, cudaStream_t st) {
    img_mul_kernel<<<grid_for((long long)n * per), 256, 0, st>>>(g, s, per, (long long)n * per);
    return cudaGetLastError();
}

cudaError_t wprep_launch(const float *W, __nv_bfloat16 *out, int cin, int cout, int flip,
                         cudaStream_t st) {
    wprep_kernel<<<grid_for(9 * cin * cout, 64), 256, 0, st>>>(W, out, cin, cout, flip);
    return cudaGetLastError();
}

cudaError_t pack_launch(const float *r, const float *ipb2, __nv_bfloat16 *img, int ns, int nt,
                        int nz, int nx, int px, long long sst, int scale_by_map, int dense,
                        cudaStream_t st) {
    const int ng = (nt + G - 1) / G, hc = (nz + 1) / 2, wc = (nx + 1) / 2;
    const int nrow = ns * ng * hc;
    if (!dense) {   // pitched rows: 16-byte loads
        pack4_kernel<<<std::min(nrow, 4096), 256, 0, st>>>(r, ipb2, img, ns, nt, ng, nz, px, sst,
                                                              hc, wc, scale_by_map);
        return cudaGetLastError();
    }
    pack_kernel<<<std::min(nrow, 4096), 256, 0, st>>>(r, ipb2, img, ns, nt, ng, nz, nx, px, sst,
                                                         hc, wc, scale_by_map, dense);
    return cudaGetLastError();
}

cudaError_t pool_launch(const __nv_bfloat16 *in, __nv_bfloat16 *out, long long n, int H, int W,
                        cudaStream_t st) {
    const int Ho = (H + 1) / 2, Wo = (W + 1) / 2;
    pool_kernel<<<grid_for(n * Ho * Wo * (C / 8)), 256, 0, st>>>(in, out, n, H, W, Ho, Wo);
    return cudaGetLastError();
}

cudaError_t upadd_launch(const __nv_bfloat16 *coarse, const __nv_bfloat16 *skip, __nv_bfloat16 *out,
                         long long n, int H, int W, cudaStream_t st) {
    upadd_kernel<<<grid_for(n * H * W * (C / 8)), 256, 0, st>>>(coarse, skip, out, n, H, W,
                                                                (H + 1) / 2, (W + 1) / 2);
    return cudaGetLastError();
}

cudaError_t mask_launch(float *g, const __nv_bfloat16 *act, __nv_bfloat16 *gb, long long n,
                        cudaStream_t st) {
    mask_kernel<<<grid_for(n), 256, 0, st>>>(g, act, gb, n);
    return cudaGetLastError();
}

cudaError_t pool_bwd_launch(float *gf, const float *gc, long long n, int H, int W, cudaStream_t st) {
    pool_bwd_kernel<<<grid_for(n * H * W * C), 256, 0, st>>>(gf, gc, n, H, W, (H + 1) / 2, (W + 1) / 2);
    return cudaGetLastError();
}

cudaError_t up_bwd_launch(const float *gf, float *gc, long long n, int H, int W, cudaStream_t st) {
    const int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    up_bwd_kernel<<<grid_for(n * Hc * Wc * C), 256, 0, st>>>(gf, gc, n, H, W, Hc, Wc);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t dw_launch(const __nv_bfloat16 *x, const __nv_bfloat16 *gy, float *part, float *gW,
                      int nimg, int H, int W, int nblk, cudaStream_t st) {
    dw_kernel<CIN, COUT><<<dim3(nblk, 9), 128, 0, st>>>(x, gy, part, nimg, H, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dw_reduce_kernel<<<grid_for(9 * CIN * COUT, 64), 256, 0, st>>>(part, gW, nblk, CIN, COUT);
    return cudaGetLastError();
}
template cudaError_t dw_launch<16, 32>(const __nv_bfloat16 *, const __nv_bfloat16 *, float *,
                                       float *, int, int, int, int, cudaStream_t);
template cudaError_t dw_launch<32, 32>(const __nv_bfloat16 *, const __nv_bfloat16 *, float *,
                                       float *, int, int, int, int, cudaStream_t);
template cudaError_t dw_launch<32, 16>(const __nv_bfloat16 *, const __nv_bfloat16 *, float *,
                                       float *, int, int, int, int, cudaStream_t);

cudaError_t bias_grad_launch(const float *g, float *gb, long long npix, int Cn, cudaStream_t st) {
    bias_grad_kernel<<<Cn, 256, 0, st>>>(g, gb, npix, Cn);
    return cudaGetLastError();
}

cudaError_t cos_loss_launch(const __nv_bfloat16 *in, const float *y, const __nv_bfloat16 *e,
                            double *dots, float *gy, long long per, int nimg, cudaStream_t st) {
    cos_dots_kernel<<<nimg, 256, 0, st>>>(in, y, e, dots, per);
    cudaError_t r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    if (gy) cos_grad_kernel<<<grid_for((long long)nimg * per), 256, 0, st>>>(in, y, e, dots, gy, per, nimg);
    return cudaGetLastError();
}

cudaError_t adam_launch(float *p, const float *g, float *m, float *v, long long n, float lr, int t,
                        cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<grid_for(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t pc_dots_launch(const float *r, const float *ap, const float *ipb2,
                           const float *y, double *part, int nblk, int ns, int nt, int nz, int nx,
                           int px, long long sst, const int *active, cudaStream_t st) {
    const int ng = (nt + G - 1) / G;
    pc_dots_kernel<<<dim3(nblk, ns), 256, 0, st>>>(r, ap, ipb2, y, part, nt, ng, nz, nx, px, sst,
                                                   (nz + 1) / 2, (nx + 1) / 2, active);
    return cudaGetLastError();
}

}  // namespace pcnet
}  // namespace esi
