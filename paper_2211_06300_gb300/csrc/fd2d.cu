// 2D propagation step (forward or time-reversed adjoint) with fused prologue/epilogue.
//
// One launch advances every shot by one time step: grid (ntx, ntz, ns), one 32 x 32
// output tile per block, 256 threads, each thread owning 4 cells of one column.  The
// input state is staged in shared memory with a 4-cell halo; cells outside the grid read
// as zero, which is the homogeneous extension under which the 8th-order Laplacian is a
// symmetric matrix (the property that makes the time-reversed run the exact adjoint).
//
// Fused work per step (each optional, selected at compile time):
//   prologue : point injection (source wavelet, or R^T e at receivers) through a per-tile
//              node list; sampling R of the *input* state from the shared tile;
//   source   : dense extended source q_n, or the CG direction update p' = r + beta p;
//   epilogue : dense output of the new state, CG product Ap = new + beta B^2 p with the
//              <p, Ap> block partial, gradient stash / correlation, saddle-point
//              correlation, on-the-fly DTFT accumulation.
#include "esi_internal.h"

namespace esi {
namespace {

// Fornberg (1988) 8th-order central weights of the second derivative, offsets 1..4
// (the centre weight is minus twice their sum, so it is folded into differences).
constexpr double W1 = 8.0 / 5.0, W2 = -1.0 / 5.0, W3 = 8.0 / 315.0, W4 = -1.0 / 560.0;

template <typename T>
__device__ __forceinline__ T lap2_tile(const T (*tl)[SW], int sz, int sx) {
    const T u = tl[sz][sx];
    T L = T(W1) * ((tl[sz][sx - 1] - u) + (tl[sz][sx + 1] - u) + (tl[sz - 1][sx] - u) +
                   (tl[sz + 1][sx] - u));
    L += T(W2) * ((tl[sz][sx - 2] - u) + (tl[sz][sx + 2] - u) + (tl[sz - 2][sx] - u) +
                  (tl[sz + 2][sx] - u));
    L += T(W3) * ((tl[sz][sx - 3] - u) + (tl[sz][sx + 3] - u) + (tl[sz - 3][sx] - u) +
                  (tl[sz + 3][sx] - u));
    L += T(W4) * ((tl[sz][sx - 4] - u) + (tl[sz][sx + 4] - u) + (tl[sz - 4][sx] - u) +
                  (tl[sz + 4][sx] - u));
    return L;
}

template <typename T>
__device__ __forceinline__ double block_sum(T v, double *red) {
    // warp level in the field precision, block level in double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x, warp = threadIdx.y;
    if (lane == 0) red[warp] = double(v);
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < BY ? red[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread (0, 0)
}

template <typename T, unsigned F>
__global__ void __launch_bounds__(BX *BY) fd2_step_kernel(const StepArgs<T> a) {
    __shared__ T tl[SH][SW];
    __shared__ T qpt[(F & F_PT) ? TZ * TX : 1];
    __shared__ double red[BY];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int s = blockIdx.z;
    if (a.active && !a.active[s]) return;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    const int tile = (s * a.ntz + blockIdx.y) * a.ntx + blockIdx.x;
    const T *cur = a.cur + (long long)s * a.sst;
    T *po = a.po + (long long)s * a.sst;

    for (int i = tid; i < SH * SW; i += BX * BY) {
        const int lz = i / SW, lx = i - lz * SW;
        const int gz = z0 - HALO + lz, gx = x0 - HALO + lx;
        T v = T(0);
        if (gz >= 0 && gz < a.nz && gx >= 0 && gx < a.nx) v = cur[(long long)gz * a.px + gx];
        tl[lz][lx] = v;
    }
    bool has_pt = false;
    if constexpr ((F & F_PT) != 0) {
        const int b = a.inj.tile_ptr[tile], e = a.inj.tile_ptr[tile + 1];
        has_pt = b < e;
        if (has_pt) {
            for (int i = tid; i < TZ * TX; i += BX * BY) qpt[i] = T(0);
            __syncthreads();
            for (int k = b + tid; k < e; k += BX * BY) {
                T sum = T(0);
                for (int c = a.inj.cptr[k]; c < a.inj.cptr[k + 1]; ++c)
                    sum += a.inj.w[c] *
                           a.inj_trace[a.inj.off0[c] + (long long)a.tin * a.inj.tstride[c]];
                qpt[a.inj.cell[k]] = sum;
            }
        }
    }
    __syncthreads();
    if constexpr ((F & F_SMP) != 0) {
        if (a.tout >= 0) {
            const int b = a.smp.tile_ptr[tile], e = a.smp.tile_ptr[tile + 1];
            const T *tf = &tl[0][0];
            for (int k = b + tid; k < e; k += BX * BY) {
                T v = T(0);
#pragma unroll
                for (int j = 0; j < 4; ++j) v += a.smp.w[k * MAXP + j] * tf[a.smp.idx[k * MAXP + j]];
                a.smp_out[a.smp.off0[k] + (long long)a.tout * a.smp.tstride[k]] = v;
            }
        }
    }

    const int gx = x0 + tx;
    const bool colok = gx < a.nx;
    const T kxv = colok ? a.kx[gx] : T(0);
    T xs = T(0), zs = T(0);
    if constexpr ((F & (F_AP | F_SAD)) != 0) {
        xs = T(a.src_pos[3 * s + 0]);
        zs = T(a.src_pos[3 * s + 2]);
    }
    T psum = T(0);
    const long long fbase = (long long)s * a.fst;
#pragma unroll
    for (int k = 0; k < RZ; ++k) {
        const int lz = ty + k * BY;
        const int gz = z0 + lz;
        if (!colok || gz >= a.nz) continue;
        const int sz = lz + HALO, sx = tx + HALO;
        const T u = tl[sz][sx];
        const T L = lap2_tile<T>(tl, sz, sx);
        const long long gi = (long long)gz * a.px + gx;
        const long long di = (long long)gz * a.nx + gx;
        T q = T(0);
        if constexpr ((F & F_EXT) != 0) q += a.ext[fbase + (long long)a.n * a.N + di];
        if constexpr ((F & F_CGP) != 0) {
            const long long vi = fbase + (long long)a.n * a.N + di;
            T pn = a.cg_r[vi];
            if (!a.cg_first) pn += T(a.cg_beta[s]) * a.cg_p[vi];
            a.cg_p[vi] = pn;
            q += pn;
        }
        T S = L + a.dx2 * q;
        if constexpr ((F & F_PT) != 0) {
            if (has_pt) S += qpt[lz * TX + tx];
        }
        const T kap = a.kz[gz] + kxv;
        const T al = T(1) / (T(1) + kap);
        const T ga = (T(1) - kap) * al;
        const T old = po[gi];
        const T nw = u + ga * (u - old) + al * a.cc[gi] * S;
        po[gi] = nw;
        if constexpr ((F & (F_AP | F_SAD)) != 0) {
            const T ex = T(gx) * a.dx - xs, ez = T(gz) * a.dx - zs;
            const T B = sqrt(ex * ex + ez * ez) + a.eps;
            const T B2 = B * B;
            if constexpr ((F & F_SAD) != 0) a.grad[(long long)s * a.N + di] += B2 * q * S;
            if constexpr ((F & F_AP) != 0) {
                const long long vi = fbase + (long long)a.nout * a.N + di;
                const T pv = a.ap_p[vi];
                const T apv = nw + a.pen * B2 * pv;
                a.ap[vi] = apv;
                psum += pv * apv;
            }
        }
        if constexpr ((F & F_STW) != 0)
            a.stash_w[((long long)a.slot_w * a.ns + s) * a.N + di] = S;
        if constexpr ((F & F_GRD) != 0)
            a.grad[(long long)s * a.N + di] +=
                nw * a.stash_r[((long long)a.slot_r * a.ns + s) * a.N + di];
        if constexpr ((F & F_OUT) != 0) a.fout[fbase + (long long)a.nout * a.N + di] = nw;
        if constexpr ((F & F_DFT) != 0) {
            for (int m = 0; m < a.nf; ++m) {
                const T c = a.twid[(a.n * a.nf + m) * 2 + 0];
                const T sn = a.twid[(a.n * a.nf + m) * 2 + 1];
                T *acc = a.dft + (((long long)s * a.nf + m) * a.N + di) * 2;
                acc[0] += nw * c;
                acc[1] += nw * sn;
            }
        }
    }
    if constexpr ((F & F_AP) != 0) {
        const double t = block_sum<T>(psum, red);
        if (tid == 0) a.dot_part[(long long)s * (a.ntx * a.ntz) + blockIdx.y * a.ntx + blockIdx.x] += t;
    }
}

template <typename T, unsigned F>
cudaError_t go(const StepArgs<T> &a, int ns, cudaStream_t st) {
    dim3 grid(a.ntx, a.ntz, ns), block(BX, BY);
    fd2_step_kernel<T, F><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
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
        return go<T, (FL)>(a, ns, st);

template <typename T>
cudaError_t launch_step2(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st) {
    switch (flags) {
        // forward modelling (point / extended / both), with and without DTFT
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

template cudaError_t launch_step2<float>(unsigned, const StepArgs<float> &, int, cudaStream_t);
template cudaError_t launch_step2<double>(unsigned, const StepArgs<double> &, int, cudaStream_t);
template cudaError_t launch_sample_global<float>(const SmpList<float> &, const float *, long long,
                                                 float *, int, cudaStream_t);
template cudaError_t launch_sample_global<double>(const SmpList<double> &, const double *,
                                                  long long, double *, int, cudaStream_t);

}  // namespace esi
