// 2D propagation step (forward or time-reversed adjoint) with fused prologue/epilogue.
//
// One launch advances every shot by one time step: grid (ntx, ntz, ns), one 64 x 32 (x, z)
// output tile per block of 256 threads.  Each thread owns one 16-byte x-vector of cells
// (4 floats or 2 doubles) in 2 (FP32) or 4 (FP64) rows, so every global stream (states,
// c, CG vectors, stash, accumulators) moves as 16-byte accesses along 128-byte rows.  The
// input state is staged in shared memory with a 4-cell halo by 16-byte loads; cells
// outside the grid read as zero, the homogeneous extension under which the 8th-order
// Laplacian is a symmetric matrix (what makes the time-reversed run the exact adjoint).
// Pad columns (nx <= x < px) of the pitched arrays: the cells of a thread's 16-byte segment
// that fall in the pad are stored as zero; segments wholly in the pad are not written, so
// kernels that read whole pitched planes skip them.
//
// Fused work per step (each optional, selected at compile time):
//   prologue : point injection (source wavelet, or R^T e at receivers) through a per-tile
//              node list; sampling R of the *input* state from the shared tile;
//   source   : dense extended source q_n (caller layout), or the CG direction update
//              p' = r + beta p (internal pitched layout);
//   epilogue : output of the new state, CG product Ap = new + beta B^2 p with the <p, Ap>
//              block partial, gradient stash / correlation, saddle-point correlation,
//              on-the-fly DTFT accumulation.
#include "esi_internal.h"

// resident blocks per SM the register allocation must allow (256 threads each)
#ifndef ESI_FD2_MINB
#define ESI_FD2_MINB 4
#endif

namespace esi {
namespace {

// Fornberg (1988) 8th-order central weights of the second derivative, offsets 0..4; in
// 2D the centre weight appears once per axis.
constexpr double W0 = -205.0 / 72.0, W1 = 8.0 / 5.0, W2 = -1.0 / 5.0, W3 = 8.0 / 315.0,
                 W4 = -1.0 / 560.0;

template <typename T>
struct alignas(16) Vec {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 3D tiled TMA load of one box into shared memory, completing on an mbarrier
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int z,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Poll the mbarrier phase with an iteration limit; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase,
                                                  long long limit) {
    for (long long i = 0; i < limit; ++i) {
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

template <typename T>
__device__ __forceinline__ Vec<T> ldv(const T *p) {
    return *reinterpret_cast<const Vec<T> *>(p);
}
template <typename T>
__device__ __forceinline__ void stv(T *p, const Vec<T> &v) {
    *reinterpret_cast<Vec<T> *>(p) = v;
}

template <typename T, unsigned F>
__global__ void __launch_bounds__(NT2, ESI_FD2_MINB) fd2_step_kernel(const __grid_constant__ StepArgs<T> a) {
    constexpr int VEC = Vec<T>::n;     // cells per thread-vector
    constexpr int TPR = TX2 / VEC;     // threads per tile row
    constexpr int RPP = NT2 / TPR;     // rows per pass
    constexpr int NP = TZ2 / RPP;      // passes
    constexpr int CPR = SW2 / VEC;     // 16-byte chunks per shared row
    __shared__ __align__(128) T tl[SH2][SW2];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ __align__(16) T qpt[(F & F_PT) ? TZ2 * TX2 : VEC];
    const int tid = threadIdx.x;
    const int s = blockIdx.z;
    if (a.active && !a.active[s]) return;
    const int x0 = blockIdx.x * TX2, z0 = blockIdx.y * TZ2;
    const int tile = (s * a.ntz + blockIdx.y) * a.ntx + blockIdx.x;
    const T *cur = a.cur + (long long)s * a.sst;
    T *po = a.po + (long long)s * a.sst;
    (void)cur;
    // stage u_n (tile + 4-cell halo) with one TMA box load; cells outside the grid are
    // zero-filled by the copy engine.  x0 - 4 is a multiple of 4 elements (16 bytes).
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int qx = tid % TPR, ry = tid / TPR;
    const int lx = qx * VEC, gx0 = x0 + lx;
    const bool colok = gx0 < a.nx;
    const long long fb = (long long)s * a.fstp;   // internal pitched fields
    const long long fd = (long long)s * a.fst;    // caller dense fields

    // Per-cell global inputs of both passes are loaded first, so that their latency
    // overlaps the staging of the shared tile instead of following the barrier.
    Vec<T> p_old[NP], p_cc[NP], p_r[NP], p_p[NP], p_g[NP], p_st[NP], p_b2[NP];
    T p_q[NP][VEC];
#pragma unroll
    for (int pz = 0; pz < NP; ++pz) {
        const int gz = z0 + ry + pz * RPP;
#pragma unroll
        for (int i = 0; i < VEC; ++i) p_q[pz][i] = T(0);
        if (!colok || gz >= a.nz) continue;
        const long long gi = (long long)gz * a.px + gx0;
        p_old[pz] = ldv(po + gi);
        p_cc[pz] = ldv(a.cc + gi);
        if constexpr ((F & F_EXT) != 0) {
            const T *e = a.ext + fd + (long long)a.n * a.N + (long long)gz * a.nx + gx0;
#pragma unroll
            for (int i = 0; i < VEC; ++i)
                if (gx0 + i < a.nx) p_q[pz][i] = e[i];
        }
        if constexpr ((F & F_CGP) != 0) {
            const long long vi = fb + (long long)a.n * a.sst + gi;
            p_r[pz] = ldv(a.cg_r + vi);
            if (!a.cg_first) p_p[pz] = ldv(a.cg_p + vi);
        }
        if constexpr ((F & F_AP) != 0) {
            p_p[pz] = ldv(a.ap_p + fb + (long long)a.nout * a.sst + gi);
            p_b2[pz] = ldv(a.pb2 + (long long)s * a.sst + gi);
        }
        if constexpr ((F & F_GRD) != 0)
            p_st[pz] = ldv(a.stash_r + ((long long)a.slot_r * a.ns + s) * a.sst + gi);
    }

    // Everything above reads only what the previous step does not write (u_{n-1} was written
    // two steps back).  Wait for the previous step, then stage its output u_n and read the
    // accumulators it updated; then let the next step's blocks start their own prologue.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)),
                     "r"((unsigned)(SH2 * SW2 * sizeof(T)))
                     : "memory");
        tma_load_3d(&tl[0][0], &a.tm, x0 - HALO, z0 - HALO, s, &bar);
    }
    if constexpr ((F & (F_GRD | F_SAD)) != 0) {
#pragma unroll
        for (int pz = 0; pz < NP; ++pz) {
            const int gz = z0 + ry + pz * RPP;
            if (colok && gz < a.nz)
                p_g[pz] = ldv(a.grad + (long long)s * a.sst + (long long)gz * a.px + gx0);
        }
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    (void)CPR;
    bool has_pt = false;
    if constexpr ((F & F_PT) != 0) {
        const int b = a.inj.tile_ptr[tile], e = a.inj.tile_ptr[tile + 1];
        has_pt = b < e;
        if (has_pt) {
            for (int i = tid; i < TZ2 * TX2; i += NT2) qpt[i] = T(0);
            __syncthreads();
            for (int k = b + tid; k < e; k += NT2) {
                T sum = T(0);
                for (int c = a.inj.cptr[k]; c < a.inj.cptr[k + 1]; ++c)
                    sum += a.inj.w[c] *
                           a.inj_trace[a.inj.off0[c] + (long long)a.tin * a.inj.tstride[c]];
                qpt[a.inj.cell[k]] = sum;
            }
        }
    }
    const bool late = !mbar_wait_bounded(&bar, 0, TMA_WAIT_LIMIT);
    if (__syncthreads_or(late)) {   // uniform: every thread of the block leaves together
        if (tid == 0) {
            atomicExch(a.dev_err, DEV_ERR_TMA_TIMEOUT);
            mbar_wait_bounded(&bar, 0, TMA_WAIT_LIMIT);  // let the copy land before leaving
        }
        return;
    }
    if constexpr ((F & F_SMP) != 0) {
        if (a.tout >= 0) {
            const int b = a.smp.tile_ptr[tile], e = a.smp.tile_ptr[tile + 1];
            const T *tf = &tl[0][0];
            for (int k = b + tid; k < e; k += NT2) {
                T v = T(0);
#pragma unroll
                for (int j = 0; j < 4; ++j) v += a.smp.w[k * MAXP + j] * tf[a.smp.idx[k * MAXP + j]];
                a.smp_out[a.smp.off0[k] + (long long)a.tout * a.smp.tstride[k]] = v;
            }
        }
    }

    T psum = T(0);
    if (colok) {
        const Vec<T> kx = ldv(a.kx + gx0);
        T xs = T(0), zs = T(0);
        if constexpr ((F & F_SAD) != 0) {
            xs = T(a.src_pos[3 * s + 0]);
            zs = T(a.src_pos[3 * s + 2]);
        }
#pragma unroll
        for (int pz = 0; pz < NP; ++pz) {
            const int lz = ry + pz * RPP;
            const int gz = z0 + lz;
            if (gz >= a.nz) break;
            const int sz = lz + HALO;
            // x neighbours: shared row segment [lx, lx + VEC + 8)
            T w[VEC + 2 * HALO];
#pragma unroll
            for (int c = 0; c < (VEC + 2 * HALO) / VEC; ++c) {
                const Vec<T> t = ldv(&tl[sz][lx + c * VEC]);
#pragma unroll
                for (int i = 0; i < VEC; ++i) w[c * VEC + i] = t.v[i];
            }
            // Laplacian sum: 2 w0 u + sum_k w_k (4 neighbours at distance k)
            T L[VEC];
#pragma unroll
            for (int i = 0; i < VEC; ++i) L[i] = T(2.0 * W0) * w[i + HALO];
            constexpr double WZ[5] = {0.0, W1, W2, W3, W4};
#pragma unroll
            for (int k = 1; k <= HALO; ++k) {
                const Vec<T> up = ldv(&tl[sz - k][lx + HALO]);
                const Vec<T> dn = ldv(&tl[sz + k][lx + HALO]);
#pragma unroll
                for (int i = 0; i < VEC; ++i)
                    L[i] += T(WZ[k]) * ((w[i + HALO - k] + w[i + HALO + k]) + (up.v[i] + dn.v[i]));
            }
            const long long gi = (long long)gz * a.px + gx0;
            const Vec<T> old = p_old[pz];
            const Vec<T> cc = p_cc[pz];
            const T kz = a.kz[gz];
            T q[VEC], S[VEC];
#pragma unroll
            for (int i = 0; i < VEC; ++i) q[i] = p_q[pz][i];
            if constexpr ((F & F_CGP) != 0) {
                const long long vi = fb + (long long)a.n * a.sst + gi;
                Vec<T> pn = p_r[pz];
                if (a.cg_pc > T(0)) {   // z = r / (pen B^2)
                    const Vec<T> ib = ldv(a.ipb2 + (long long)s * a.sst + gi);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) pn.v[i] *= ib.v[i];
                    if (a.pc_y) {   // + theta x the learned coarse correction of this time sample
                        // (planes [s][pc_ng * 16][pc_hc][pc_wc])
                        const float *yr = a.pc_y +
                            (((long long)s * a.pc_ng * 16 + a.n) * a.pc_hc + gz / 2) * a.pc_wc;
                        const T th = T(a.pc_theta[s]);
#pragma unroll
                        for (int i = 0; i < VEC; ++i)
                            if (gx0 + i < a.nx) pn.v[i] += th * T(yr[(gx0 + i) / 2]);
                    }
                }
                if (!a.cg_first) {
                    const T b = T(a.cg_beta[s]);
#pragma unroll
                    for (int i = 0; i < VEC; ++i) pn.v[i] += b * p_p[pz].v[i];
                }
                stv(a.cg_p + vi, pn);
#pragma unroll
                for (int i = 0; i < VEC; ++i) q[i] += pn.v[i];
            }
#pragma unroll
            for (int i = 0; i < VEC; ++i) S[i] = L[i] + a.dx2 * q[i];
            if constexpr ((F & F_PT) != 0) {
                if (has_pt) {
#pragma unroll
                    for (int i = 0; i < VEC; ++i) S[i] += qpt[lz * TX2 + lx + i];
                }
            }
            Vec<T> nw;
            bool sponge = kz != T(0);
#pragma unroll
            for (int i = 0; i < VEC; ++i) sponge |= kx.v[i] != T(0);
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
            stv(po + gi, nw);
            if constexpr ((F & F_SAD) != 0) {
                T B2[VEC];
                const T ez = T(gz) * a.dx - zs;
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    const T ex = T(gx0 + i) * a.dx - xs;
                    const T B = a.unit_b ? T(1) : sqrt(ex * ex + ez * ez) + a.eps;
                    B2[i] = B * B;
                }
                {
                    Vec<T> gv = p_g[pz];
#pragma unroll
                    for (int i = 0; i < VEC; ++i) gv.v[i] += B2[i] * q[i] * S[i];
                    stv(a.grad + (long long)s * a.sst + gi, gv);
                }
            }
            if constexpr ((F & F_AP) != 0) {   // A p = S^T S p + pen B^2 p
                const long long vi = fb + (long long)a.nout * a.sst + gi;
                const Vec<T> pv = p_p[pz];
                const Vec<T> b2 = p_b2[pz];
                Vec<T> av;
#pragma unroll
                for (int i = 0; i < VEC; ++i) {
                    av.v[i] = nw.v[i] + b2.v[i] * pv.v[i];
                    psum += pv.v[i] * av.v[i];
                }
                stv(a.ap + vi, av);
            }
            if constexpr ((F & F_STW) != 0) {
                Vec<T> sv;
#pragma unroll
                for (int i = 0; i < VEC; ++i) sv.v[i] = (gx0 + i < a.nx) ? S[i] : T(0);
                stv(a.stash_w + ((long long)a.slot_w * a.ns + s) * a.sst + gi, sv);
            }
            if constexpr ((F & F_GRD) != 0) {
                Vec<T> gv = p_g[pz];
#pragma unroll
                for (int i = 0; i < VEC; ++i) gv.v[i] += nw.v[i] * p_st[pz].v[i];
                stv(a.grad + (long long)s * a.sst + gi, gv);
            }
            if constexpr ((F & F_OUT) != 0) {
                T *o = a.fout + (long long)s * a.ofst + (long long)a.nout * a.oplane +
                       (long long)gz * a.opx + gx0;
                if (a.opx == a.px) {
                    stv(o, nw);
                } else {
#pragma unroll
                    for (int i = 0; i < VEC; ++i)
                        if (gx0 + i < a.nx) o[i] = nw.v[i];
                }
            }
            if constexpr ((F & F_DFT) != 0)   // the DTFT's block stash (slot n - n0)
                stv(a.stash_w + ((long long)a.slot_w * a.ns + s) * a.sst + gi, nw);
        }
    }
    if constexpr ((F & F_AP) != 0) {
        // one partial per warp (no block-wide wait at the end): dot_part[shot][tile][warp],
        // accumulated over the time steps.  Each slot has one writer per step and the steps
        // of a loop complete in order, so the sums are deterministic.
        T v = psum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0)   // a reduction without return: no load latency at the block's end
            atomicAdd(&a.dot_part[((long long)s * (a.ntx * a.ntz) + blockIdx.y * a.ntx + blockIdx.x) *
                                  (NT2 / 32) + (tid >> 5)], double(v));
    }
}

// chained: the previous launch on the stream is the previous step of the same loop, so the
// grid may start (programmatic dependent launch) while that step drains: its prologue reads
// only what that step does not write, and it waits for it before staging u_n.
template <typename T, unsigned F>
cudaError_t go(const StepArgs<T> &a, int ns, cudaStream_t st, bool chained) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ntx, a.ntz, ns);
    cfg.blockDim = dim3(NT2);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fd2_step_kernel<T, F>, a);
}

template <typename T>
__global__ void sample_global_kernel(const SmpList<T> l, const T *state, long long sst, T *out,
                                     int tout) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= l.nrec) return;
    const T *u = state + (long long)l.shot[r] * sst;
    T v = T(0);
#pragma unroll
    for (int j = 0; j < MAXP; ++j) v += l.w[r * MAXP + j] * u[l.gidx[r * MAXP + j]];
    out[l.off0[r] + (long long)tout * l.tstride[r]] = v;
}

}  // namespace

#define ESI_CASE(FL)        \
    case (FL):              \
        return go<T, (FL)>(a, ns, st, chained);

template <typename T>
cudaError_t launch_step2(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st,
                         bool chained) {
    switch (flags) {
        // forward modelling (point / extended / both), with and without DTFT; the
        // F_PT | F_SMP variant also serves the adjoint with the wavelet output only
        ESI_CASE(F_PT | F_SMP)
        ESI_CASE(F_EXT | F_SMP)
        ESI_CASE(F_EXT | F_PT | F_SMP)
        ESI_CASE(F_PT | F_SMP | F_DFT)
        ESI_CASE(F_EXT | F_SMP | F_DFT)
        ESI_CASE(F_EXT | F_PT | F_SMP | F_DFT)
        // CG product, forward half
        ESI_CASE(F_CGP | F_SMP)
        // gradient recompute segments
        ESI_CASE(F_PT | F_STW)
        ESI_CASE(F_EXT | F_STW)
        ESI_CASE(F_EXT | F_PT | F_STW)
        // saddle-point gradient
        ESI_CASE(F_EXT | F_SAD)
        ESI_CASE(F_EXT | F_PT | F_SAD)   // WRI: u = A^{-1}(f + q)
        ESI_CASE(F_EXT | F_SMP | F_SAD)  // ... with the traces for the objective
        ESI_CASE(F_EXT | F_PT | F_SMP | F_SAD)
        // adjoint modelling
        ESI_CASE(F_PT)
        ESI_CASE(F_PT | F_OUT)
        ESI_CASE(F_PT | F_OUT | F_SMP)
        ESI_CASE(F_PT | F_AP)
        ESI_CASE(F_PT | F_GRD)
        default:
            return cudaErrorInvalidValue;
    }
}
#undef ESI_CASE

template <typename T>
cudaError_t launch_sample_global(const SmpList<T> &l, const T *state, long long sst, T *out,
                                 int tout, cudaStream_t st) {
    if (l.nrec == 0) return cudaSuccess;
    const int th = 128;
    sample_global_kernel<T><<<(l.nrec + th - 1) / th, th, 0, st>>>(l, state, sst, out, tout);
    return cudaGetLastError();
}

template cudaError_t launch_step2<float>(unsigned, const StepArgs<float> &, int, cudaStream_t, bool);
template cudaError_t launch_step2<double>(unsigned, const StepArgs<double> &, int, cudaStream_t, bool);
template cudaError_t launch_sample_global<float>(const SmpList<float> &, const float *, long long,
                                                 float *, int, cudaStream_t);
template cudaError_t launch_sample_global<double>(const SmpList<double> &, const double *,
                                                  long long, double *, int, cudaStream_t);

}  // namespace esi
