// 3D propagation step with register marching along z (the slow axis).
//
// A block owns a 32 x 16 column tile of the xy plane and a chunk of ZCH3 planes.  Each
// thread keeps the 9 values u(z-4 .. z+4) of its own column in registers; the plane z
// is staged in shared memory with a 4-cell x/y halo for the in-plane neighbours.  So
// every cell of the input state is read from global memory once per chunk by its owner
// (plus the halo, mostly served by L2), the older state and c once, and the new state
// written once.  Receiver sampling is done by a separate gather launch (trilinear
// points straddle two planes); point injection walks a per-tile node list sorted by z.
#include "esi_internal.h"

namespace esi {

constexpr int ZCH3 = 64;  // planes per block (z chunk)

namespace {

constexpr double W1 = 8.0 / 5.0, W2 = -1.0 / 5.0, W3 = 8.0 / 315.0, W4 = -1.0 / 560.0;

template <typename T, unsigned F>
__global__ void __launch_bounds__(TX3 *TY3) fd3_step_kernel(const StepArgs<T> a, int nzc) {
    __shared__ T pl[SH3][SW3];
    __shared__ double red[TX3 * TY3 / 32];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX3 + tx;
    const int s = blockIdx.z / nzc, zc = blockIdx.z - s * nzc;
    if (a.active && !a.active[s]) return;
    const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool colok = gx < a.nx && gy < a.ny;
    const int zb = zc * ZCH3, ze = min(a.nz, zb + ZCH3);
    const long long plane = (long long)a.ny * a.px;
    const T *cur = a.cur + (long long)s * a.sst;
    T *po = a.po + (long long)s * a.sst;
    const long long col = (long long)gy * a.px + gx;
    const int tile = ((s * nzc + zc) * a.nty + blockIdx.y) * a.ntx + blockIdx.x;

    T q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int z = zb - HALO + k;
        q[k] = (colok && z >= 0 && z < a.nz) ? cur[z * plane + col] : T(0);
    }
    const T kxy = colok ? a.kx[gx] + a.ky[gy] : T(0);
    T xs = T(0), ys = T(0), zs = T(0);
    if constexpr ((F & (F_AP | F_SAD | F_CGP)) != 0) {
        xs = T(a.src_pos[3 * s + 0]);
        ys = T(a.src_pos[3 * s + 1]);
        zs = T(a.src_pos[3 * s + 2]);
    }
    int ip = 0, ie = 0;
    if constexpr ((F & F_PT) != 0) {
        ip = a.inj.tile_ptr[tile];
        ie = a.inj.tile_ptr[tile + 1];
    }
    T psum = T(0);
    const long long fbase = (long long)s * a.fst;    // caller dense fields
    const long long fb = (long long)s * a.fstp;      // internal pitched fields
    const long long dcol = (long long)gy * a.nx + gx;

    for (int z = zb; z < ze; ++z) {
        pl[ty + HALO][tx + HALO] = q[HALO];
        for (int i = tid; i < SH3 * SW3; i += TX3 * TY3) {
            const int ly = i / SW3, lx = i - ly * SW3;
            if (ly >= HALO && ly < TY3 + HALO && lx >= HALO && lx < TX3 + HALO) continue;
            const int hy = y0 - HALO + ly, hx = x0 - HALO + lx;
            T v = T(0);
            if (hy >= 0 && hy < a.ny && hx >= 0 && hx < a.nx)
                v = cur[z * plane + (long long)hy * a.px + hx];
            pl[ly][lx] = v;
        }
        __syncthreads();
        if (colok) {
            const int sy = ty + HALO, sx = tx + HALO;
            const T u = q[HALO];
            T L = T(W1) * ((pl[sy][sx - 1] - u) + (pl[sy][sx + 1] - u) + (pl[sy - 1][sx] - u) +
                           (pl[sy + 1][sx] - u) + (q[3] - u) + (q[5] - u));
            L += T(W2) * ((pl[sy][sx - 2] - u) + (pl[sy][sx + 2] - u) + (pl[sy - 2][sx] - u) +
                          (pl[sy + 2][sx] - u) + (q[2] - u) + (q[6] - u));
            L += T(W3) * ((pl[sy][sx - 3] - u) + (pl[sy][sx + 3] - u) + (pl[sy - 3][sx] - u) +
                          (pl[sy + 3][sx] - u) + (q[1] - u) + (q[7] - u));
            L += T(W4) * ((pl[sy][sx - 4] - u) + (pl[sy][sx + 4] - u) + (pl[sy - 4][sx] - u) +
                          (pl[sy + 4][sx] - u) + (q[0] - u) + (q[8] - u));
            const long long gi = z * plane + col;
            const long long di = (long long)z * a.ny * a.nx + dcol;
            T src = T(0);
            if constexpr ((F & F_EXT) != 0) src += a.ext[fbase + (long long)a.n * a.N + di];
            if constexpr ((F & F_CGP) != 0) {
                const long long vi = fb + (long long)a.n * a.sst + gi;
                T pn = a.cg_r[vi];
                if (a.cg_pc > T(0)) pn *= a.ipb2[(long long)s * a.sst + gi];   // z = r / (pen B^2)
                if (!a.cg_first) pn += T(a.cg_beta[s]) * a.cg_p[vi];
                a.cg_p[vi] = pn;
                src += pn;
            }
            T S = L + a.dx2 * src;
            if constexpr ((F & F_PT) != 0) {
                // entries sorted by z: consume those of this plane
                while (ip < ie) {
                    const int cell = a.inj.cell[ip];
                    const int cz = cell / (TX3 * TY3);
                    if (cz != z) break;
                    const int rem = cell - cz * (TX3 * TY3);
                    if (rem == ty * TX3 + tx) {
                        T sum = T(0);
                        for (int c = a.inj.cptr[ip]; c < a.inj.cptr[ip + 1]; ++c)
                            sum += a.inj.w[c] *
                                   a.inj_trace[a.inj.off0[c] + (long long)a.tin * a.inj.tstride[c]];
                        S += sum;
                    }
                    ++ip;
                }
            }
            const T kap = a.kz[z] + kxy;
            const T al = T(1) / (T(1) + kap);
            const T ga = (T(1) - kap) * al;
            const T old = po[gi];
            const T nw = u + ga * (u - old) + al * a.cc[gi] * S;
            po[gi] = nw;
            if constexpr ((F & F_SAD) != 0) {
                const T ex = T(gx) * a.dx - xs, ey = T(gy) * a.dx - ys, ez = T(z) * a.dx - zs;
                const T B = sqrt(ex * ex + ey * ey + ez * ez) + a.eps;
                a.grad[(long long)s * a.sst + gi] += B * B * src * S;
            }
            if constexpr ((F & F_AP) != 0) {   // A p = S^T S p + pen B^2 p
                const long long vi = fb + (long long)a.nout * a.sst + gi;
                const T pv = a.ap_p[vi];
                const T apv = nw + a.pb2[(long long)s * a.sst + gi] * pv;
                a.ap[vi] = apv;
                psum += pv * apv;
            }
            if constexpr ((F & F_STW) != 0)
                a.stash_w[((long long)a.slot_w * a.ns + s) * a.sst + gi] = S;
            if constexpr ((F & F_GRD) != 0)
                a.grad[(long long)s * a.sst + gi] +=
                    nw * a.stash_r[((long long)a.slot_r * a.ns + s) * a.sst + gi];
            if constexpr ((F & F_OUT) != 0)
                a.fout[(long long)s * a.ofst + (long long)a.nout * a.oplane +
                       ((long long)z * a.ny + gy) * a.opx + gx] = nw;
            if constexpr ((F & F_DFT) != 0) {
                for (int m = 0; m < a.nf; ++m) {
                    const T c = a.twid[(a.n * a.nf + m) * 2 + 0];
                    const T sn = a.twid[(a.n * a.nf + m) * 2 + 1];
                    T *acc = a.dft + (((long long)s * a.nf + m) * a.sst + gi) * 2;
                    acc[0] += nw * c;
                    acc[1] += nw * sn;
                }
            }
        } else if constexpr ((F & F_PT) != 0) {
            while (ip < ie && a.inj.cell[ip] / (TX3 * TY3) == z) ++ip;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
        const int zn = z + HALO + 1;
        q[8] = (colok && zn < a.nz) ? cur[zn * plane + col] : T(0);
    }
    if constexpr ((F & F_AP) != 0) {
        T v = psum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[tid >> 5] = double(v);
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < TX3 * TY3 / 32; ++w) t += red[w];
            const long long nblk = (long long)a.ntx * a.nty * nzc;
            a.dot_part[s * nblk + ((long long)zc * a.nty + blockIdx.y) * a.ntx + blockIdx.x] += t;
        }
    }
}

template <typename T, unsigned F>
cudaError_t go(const StepArgs<T> &a, int ns, cudaStream_t st) {
    const int nzc = (a.nz + ZCH3 - 1) / ZCH3;
    dim3 grid(a.ntx, a.nty, ns * nzc), block(TX3, TY3);
    fd3_step_kernel<T, F><<<grid, block, 0, st>>>(a, nzc);
    return cudaGetLastError();
}

}  // namespace

#define ESI_CASE(FL)        \
    case (FL):              \
        return go<T, (FL)>(a, ns, st);

template <typename T>
cudaError_t launch_step3(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st) {
    switch (flags) {
        ESI_CASE(F_PT)
        ESI_CASE(F_EXT)
        ESI_CASE(F_EXT | F_PT)
        ESI_CASE(F_PT | F_DFT)
        ESI_CASE(F_EXT | F_DFT)
        ESI_CASE(F_EXT | F_PT | F_DFT)
        ESI_CASE(F_CGP)
        ESI_CASE(F_PT | F_STW)
        ESI_CASE(F_EXT | F_STW)
        ESI_CASE(F_EXT | F_PT | F_STW)
        ESI_CASE(F_EXT | F_SAD)
        ESI_CASE(F_PT | F_OUT)
        ESI_CASE(F_PT | F_AP)
        ESI_CASE(F_PT | F_GRD)
        default:
            return cudaErrorInvalidValue;
    }
}
#undef ESI_CASE

template cudaError_t launch_step3<float>(unsigned, const StepArgs<float> &, int, cudaStream_t);
template cudaError_t launch_step3<double>(unsigned, const StepArgs<double> &, int, cudaStream_t);

}  // namespace esi
