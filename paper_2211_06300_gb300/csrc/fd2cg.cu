// The two halves of the ESI normal-equation product (the CG section's matrix-vector product:
// one forward modelling with p as the extended source, one adjoint modelling of its traces
// plus lambda B^2 p) as persistent, TMA-fed 2D step kernels.
//
//   forward half (F_CGP | F_SMP): p_n = z_n + beta p_n, z = r (or r / (lambda B^2), plus the
//     learned correction), u_{n+1} = step(u_n, u_{n-1}; source p_n), traces of u_n;
//   adjoint half (F_PT | F_AP): mu_{n+1} = step(mu_n, mu_{n-1}; traces), A p = mu + lambda B^2 p
//     with per-warp partials of <p, A p>.
//
// Each block loops over 64 x 32 tiles (all shots' tiles of the time step, inactive shots
// skipped).  Every input of a tile -- u_n with its 4-cell halo, u_{n-1}, c and the tile's
// interior boxes of the CG streams (r, 1/(lambda B^2), p or p, lambda B^2) -- arrives by TMA
// in one of two shared-memory stages; while the block computes tile i from its stage, the
// copies of tile i + 1 are in flight into the other.  So the warps read only shared memory,
// the block keeps two tiles of bytes in flight, and no per-tile global-load latency remains
// on the path.  Outputs (u_{n+1}, p or A p) are 16-byte stores.
#include "esi_internal.h"

namespace esi {

namespace {

constexpr double W0 = -205.0 / 72.0, W1 = 8.0 / 5.0, W2 = -1.0 / 5.0, W3 = 8.0 / 315.0,
                 W4 = -1.0 / 560.0;

template <typename T>
struct alignas(16) V {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};
template <typename T>
__device__ __forceinline__ V<T> ld16(const T *p) {
    return *reinterpret_cast<const V<T> *>(p);
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const V<T> &v) {
    *reinterpret_cast<V<T> *>(p) = v;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tma2(void *dst, const CUtensorMap *tm, int x, int y,
                                     unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                     unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma4(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                     int w, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(w),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool wait_bounded(unsigned long long *bar, unsigned phase) {
    for (long long i = 0; i < TMA_WAIT_LIMIT; ++i) {
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

// one stage: u_n with halo, u_{n-1}, c, and the CG streams a (r | p), b (1/(lambda B^2) |
// lambda B^2), c2 (p, forward half only)
template <typename T, bool FWD>
struct Stage {
    T u[SH2][SW2];
    T old[TZ2][TX2];
    T c[TZ2][TX2];
    T a[TZ2][TX2];
    T b[TZ2][TX2];
    T c2[FWD ? TZ2 : 1][TX2];
};
static_assert(sizeof(Stage<float, true>) % 128 == 0 && sizeof(Stage<float, false>) % 128 == 0 &&
                  (SH2 * SW2 * 4) % 128 == 0 && (TZ2 * TX2 * 4) % 128 == 0,
              "stage buffers must keep the 128-byte alignment of TMA destinations");

template <typename T, bool FWD>
constexpr int cg_smem() {
    return 2 * (int)sizeof(Stage<T, FWD>) + (FWD ? 0 : TZ2 * TX2 * (int)sizeof(T)) + 128;
}

template <typename T, bool FWD>
__global__ void __launch_bounds__(NT2, 1) fd2_cg_kernel(const __grid_constant__ StepArgs<T> a,
                                                        int total) {
    constexpr int VEC = V<T>::n;
    constexpr int TPR = TX2 / VEC, RPP = NT2 / TPR, NP = TZ2 / RPP;
    extern __shared__ unsigned char smraw[];
    unsigned char *base = smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u);
    Stage<T, FWD> *stage = reinterpret_cast<Stage<T, FWD> *>(base);
    T *qpt = reinterpret_cast<T *>(base + 2 * sizeof(Stage<T, FWD>));   // adjoint: injected traces
    __shared__ __align__(8) unsigned long long full[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tps = a.ntx * a.ntz;   // tiles per shot
    const int qx = tid % TPR, ry = tid / TPR;
    const int lx = qx * VEC;
    const bool use_b = FWD ? a.cg_pc > T(0) : true;
    const bool use_c2 = FWD && !a.cg_first;
    const unsigned bytes = (unsigned)sizeof(T) *
                           (SH2 * SW2 + (3 + (use_b ? 1 : 0) + (use_c2 ? 1 : 0)) * TZ2 * TX2);
    if (tid == 0) {
        for (int k = 0; k < 2; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[k])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto next = [&](int t) {   // the first tile >= t of this block whose shot is active
        while (t < total && a.active && !a.active[t / tps]) t += gridDim.x;
        return t;
    };
    const int tv = FWD ? a.n : a.nout;   // time index of the space-time streams
    auto issue = [&](int t, int k) {     // thread 0: all boxes of tile t into stage k
        const int s = t / tps, rem = t - s * tps;
        const int x0 = (rem % a.ntx) * TX2, z0 = (rem / a.ntx) * TZ2;
        Stage<T, FWD> &st = stage[k];
        unsigned long long *bar = &full[k];
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"(bytes)
                     : "memory");
        // x0 - 4 and x0 are multiples of 4 elements (16 bytes)
        tma3(&st.u[0][0], &a.tm, x0 - HALO, z0 - HALO, s, bar);
        tma3(&st.old[0][0], &a.tm_old, x0, z0, s, bar);
        tma2(&st.c[0][0], &a.tm_cc, x0, z0, bar);
        tma4(&st.a[0][0], &a.tm_a, x0, z0, tv, s, bar);
        if (use_b) tma3(&st.b[0][0], &a.tm_b, x0, z0, s, bar);
        if constexpr (FWD) {
            if (use_c2) tma4(&st.c2[0][0], &a.tm_c, x0, z0, tv, s, bar);
        }
    };
    int t = next(blockIdx.x);
    if (tid == 0 && t < total) issue(t, 0);
    bool late = false, failed = false, next_pending = false;
    int it = 0;
    for (; t < total; ++it) {
        const int k = it & 1;
        const int tn = next(t + gridDim.x);
        next_pending = tn < total;
        if (tid == 0 && next_pending) issue(tn, k ^ 1);   // stage k ^ 1 was released last round
        const int s = t / tps, rem = t - s * tps;
        const int x0 = (rem % a.ntx) * TX2, z0 = (rem / a.ntx) * TZ2;
        const int gx0 = x0 + lx;
        const bool colok = gx0 < a.nx;
        T *po = a.po + (long long)s * a.sst;
        const long long fb = (long long)s * a.fstp;
        bool has_pt = false;
        if constexpr (!FWD) {   // the traces injected in this tile (adjoint sources)
            const int b = a.inj.tile_ptr[t], e = a.inj.tile_ptr[t + 1];
            has_pt = b < e;
            if (has_pt) {
                for (int i = tid; i < TZ2 * TX2; i += NT2) qpt[i] = T(0);
                __syncthreads();
                for (int j = b + tid; j < e; j += NT2) {
                    T sum = T(0);
                    for (int c = a.inj.cptr[j]; c < a.inj.cptr[j + 1]; ++c)
                        sum += a.inj.w[c] *
                               a.inj_trace[a.inj.off0[c] + (long long)a.tin * a.inj.tstride[c]];
                    qpt[a.inj.cell[j]] = sum;
                }
            }
        }
        late |= !wait_bounded(&full[k], (unsigned)(it >> 1) & 1u);
        if (__syncthreads_or(late)) {
            failed = true;
            break;
        }
        const Stage<T, FWD> &st = stage[k];
        if constexpr (FWD) {   // traces of u_n from the staged tile
            if (a.tout >= 0) {
                const int b = a.smp.tile_ptr[t], e = a.smp.tile_ptr[t + 1];
                const T *tf = &st.u[0][0];
                for (int j = b + tid; j < e; j += NT2) {
                    T v = T(0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) v += a.smp.w[j * MAXP + q] * tf[a.smp.idx[j * MAXP + q]];
                    a.smp_out[a.smp.off0[j] + (long long)a.tout * a.smp.tstride[j]] = v;
                }
            }
        }
        T psum = T(0);
        if (colok) {
            const V<T> kx = ld16(a.kx + gx0);
            const T beta = FWD && !a.cg_first ? T(a.cg_beta[s]) : T(0);
            T th = T(0);
            if constexpr (FWD) {
                if (a.pc_y) th = T(a.pc_theta[s]);
            }
            (void)th;
#pragma unroll
            for (int pz = 0; pz < NP; ++pz) {
                const int lz = ry + pz * RPP;
                const int gz = z0 + lz;
                if (gz >= a.nz) break;
                const int sz = lz + HALO;
                T w[VEC + 2 * HALO];
#pragma unroll
                for (int c = 0; c < (VEC + 2 * HALO) / VEC; ++c) {
                    const V<T> tv2 = ld16(&st.u[sz][lx + c * VEC]);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) w[c * VEC + i] = tv2.v[i];
                }
                T L[VEC];
#pragma unroll
                for (int i = 0; i < VEC; ++i) L[i] = T(2.0 * W0) * w[i + HALO];
                constexpr double WZ[5] = {0.0, W1, W2, W3, W4};
#pragma unroll
                for (int d = 1; d <= HALO; ++d) {
                    const V<T> up = ld16(&st.u[sz - d][lx + HALO]);
                    const V<T> dn = ld16(&st.u[sz + d][lx + HALO]);
#pragma unroll
                    for (int i = 0; i < VEC; ++i)
                        L[i] += T(WZ[d]) * ((w[i + HALO - d] + w[i + HALO + d]) + (up.v[i] + dn.v[i]));
                }
                const long long gi = (long long)gz * a.px + gx0;
                const long long vi = fb + (long long)tv * a.sst + gi;
                const V<T> old = ld16(&st.old[lz][lx]);
                const V<T> cc = ld16(&st.c[lz][lx]);
                T S[VEC];
                if constexpr (FWD) {
                    V<T> pn = ld16(&st.a[lz][lx]);
                    if (use_b) {   // z = r / (pen B^2) (+ the learned correction)
                        const V<T> ib = ld16(&st.b[lz][lx]);
#pragma unroll
                        for (int i = 0; i < VEC; ++i) pn.v[i] *= ib.v[i];
                        if (a.pc_y) {
                            const float *yr = a.pc_y +
                                (((long long)s * a.pc_ng * 16 + a.n) * a.pc_hc + gz / 2) * a.pc_wc;
#pragma unroll
                            for (int i = 0; i < VEC; ++i)
                                if (gx0 + i < a.nx) pn.v[i] += th * T(yr[(gx0 + i) / 2]);
                        }
                    }
                    if (use_c2) {
                        const V<T> pp = ld16(&st.c2[lz][lx]);
#pragma unroll
                        for (int i = 0; i < VEC; ++i) pn.v[i] += beta * pp.v[i];
                    }
                    st16(a.cg_p + vi, pn);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) S[i] = L[i] + a.dx2 * pn.v[i];
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) S[i] = L[i];
                    if (has_pt) {
#pragma unroll
                        for (int i = 0; i < VEC; ++i) S[i] += qpt[lz * TX2 + lx + i];
                    }
                }
                const T kz = a.kz[gz];
                bool sponge = kz != T(0);
#pragma unroll
                for (int i = 0; i < VEC; ++i) sponge |= kx.v[i] != T(0);
                V<T> nw;
                if (sponge) {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        const T kap = kz + kx.v[i];
                        const T al = T(1) / (T(1) + kap);
                        const T ga = (T(1) - kap) * al;
                        const T u = w[i + HALO];
                        nw.v[i] = u + ga * (u - old.v[i]) + al * cc.v[i] * S[i];
                    }
                } else {   // interior: alpha = gamma = 1
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        const T u = w[i + HALO];
                        nw.v[i] = u + (u - old.v[i]) + cc.v[i] * S[i];
                    }
                }
#pragma unroll
                for (int i = 0; i < VEC; ++i)
                    if (gx0 + i >= a.nx) nw.v[i] = T(0);   // pad columns stay zero
                st16(po + gi, nw);
                if constexpr (!FWD) {   // A p = S^T S p + pen B^2 p
                    const V<T> pv = ld16(&st.a[lz][lx]);
                    const V<T> pb = ld16(&st.b[lz][lx]);
                    V<T> av;
#pragma unroll
                    for (int i = 0; i < VEC; ++i) {
                        av.v[i] = nw.v[i] + pb.v[i] * pv.v[i];
                        psum += pv.v[i] * av.v[i];
                    }
                    st16(a.ap + vi, av);
                }
            }
        }
        if constexpr (!FWD) {   // per-warp partial of <p, A p>: dot_part[shot][tile][warp]
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) psum += __shfl_xor_sync(0xffffffffu, psum, o);
            if (lane == 0) a.dot_part[((long long)s * tps + rem) * (NT2 / 32) + warp] += double(psum);
        }
        __syncthreads();   // stage k is free for the copies of tile it + 2
        t = tn;
    }
    if (failed && tid == 0) {
        atomicExch(a.dev_err, DEV_ERR_TMA_TIMEOUT);
        // let the copies in flight land before the block's shared memory is released: this
        // tile's stage, and the next tile's if it was issued
        wait_bounded(&full[it & 1], (unsigned)(it >> 1) & 1u);
        if (next_pending) wait_bounded(&full[(it + 1) & 1], (unsigned)((it + 1) >> 1) & 1u);
    }
    __syncthreads();
}

int sm_count() {
    static PerDevice cache;
    int n = 0;
    const cudaError_t e = per_device(cache, &n, [](int *v) {
        int dev = 0;
        cudaError_t r = cudaGetDevice(&dev);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev);
        return r;
    });
    return e == cudaSuccess && n > 0 ? n : 152;   // GB300's count if the query failed
}

template <typename T, bool FWD>
cudaError_t go_cg(const StepArgs<T> &a, int ns, cudaStream_t st) {
    auto kern = fd2_cg_kernel<T, FWD>;
    static PerDevice cache;
    int per_sm = 0;
    cudaError_t e = per_device(cache, &per_sm, [kern](int *v) {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             cg_smem<T, FWD>());
        if (r != cudaSuccess) return r;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, kern, NT2, cg_smem<T, FWD>());
        *v = std::max(1, *v);
        return r;
    });
    if (e != cudaSuccess) return e;
    const int total = ns * a.ntx * a.ntz;
    const int grid = std::min(total, sm_count() * per_sm);
    kern<<<grid, NT2, cg_smem<T, FWD>(), st>>>(a, total);
    return cudaGetLastError();
}

}  // namespace

template <typename T>
cudaError_t launch_step2_cg(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st) {
    if (flags == (F_CGP | F_SMP)) return go_cg<T, true>(a, ns, st);
    if (flags == (F_PT | F_AP)) return go_cg<T, false>(a, ns, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_step2_cg<float>(unsigned, const StepArgs<float> &, int, cudaStream_t);
template cudaError_t launch_step2_cg<double>(unsigned, const StepArgs<double> &, int, cudaStream_t);

}  // namespace esi
