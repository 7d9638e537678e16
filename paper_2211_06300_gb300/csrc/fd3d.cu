// 3D propagation step: TMA-staged xy planes, register marching along z (the slow axis).
//
// A block owns a 32 x 16 column tile of the xy plane and a chunk of ZCH3 planes.  The
// planes of its column tile, each with a 4-cell x/y halo, arrive by TMA (one 40 x 24 box per
// plane, zero-filled outside the grid) in a ring of RING3 shared-memory slots, together with
// the tile interior of the older state and of c.  One producer warp keeps the ring filled
// (a slot is refilled once every consumer warp has released it on an mbarrier), so the
// consumer warps never meet at a block-wide barrier while marching.  A consumer thread owns
// one 16-byte row segment (4 FP32 or 2 FP64 cells) and keeps the 9 values u(z-4 .. z+4) of
// those cells in registers, refilled from the ring.  So every cell of the input state
// crosses from HBM once per chunk (plus the z halo of the chunk and the xy halo, mostly
// served by L2), the older state and c once, and the new state is written once, with no
// global-load latency on the marching path.  Receiver sampling of the input state is a
// gather from global memory by the consumer threads of the block whose tile and chunk hold
// the receiver's base node, issued while the first planes are in flight (trilinear points
// straddle two planes, possibly two chunks); point injection walks a per-tile node list
// sorted by z.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "esi_internal.h"

namespace esi {

namespace {

// Fornberg (1988) 8th-order central weights of the second derivative, offsets 0..4; in 3D
// the centre weight appears once per axis.
constexpr double W0 = -205.0 / 72.0, W1 = 8.0 / 5.0, W2 = -1.0 / 5.0, W3 = 8.0 / 315.0,
                 W4 = -1.0 / 560.0;

template <typename T>
struct alignas(16) Vec3 {
    static constexpr int n = 16 / sizeof(T);
    T v[n];
};
template <typename T>
__device__ __forceinline__ Vec3<T> ldv3(const T *p) {
    return *reinterpret_cast<const Vec3<T> *>(p);
}
template <typename T>
__device__ __forceinline__ void stv3(T *p, const Vec3<T> &v) {
    *reinterpret_cast<Vec3<T> *>(p) = v;
}

template <typename T>
__host__ __device__ constexpr int consumers3() {   // one 16-byte row segment of the tile per consumer thread
    return TX3 * TY3 / Vec3<T>::n;
}
template <typename T>
__host__ __device__ constexpr int block3() {     // + one producer warp
    return consumers3<T>() + 32;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 4D tiled TMA load (x, y, z, shot) of one plane box, completing on an mbarrier
__device__ __forceinline__ void tma_load_plane(void *dst, const CUtensorMap *tm, int x, int y,
                                               int z, int s, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(s),
        "r"(smem_u32(bar))
        : "memory");
}

// Poll the mbarrier phase with an iteration limit; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned phase) {
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

// one ring slot: the halo box of u_n, then the interior boxes of u_{n-1} and c
template <typename T>
struct Slot3 {
    T u[SH3][SW3];
    T old[TY3][TX3];
    T c[TY3][TX3];
};
static_assert(sizeof(Slot3<float>) % 128 == 0 && sizeof(Slot3<double>) % 128 == 0,
              "ring slots must keep the 128-byte alignment of TMA destinations");

// the marching step i holds planes i + 4 (its xy plane) .. i + 9 (the queue refill): six
// slots, plus at least one being filled
static_assert(RING3 >= 2 * HALO - 1, "the plane ring needs room for the live planes and one more");

template <typename T>
constexpr int ring_bytes() {
    return RING3 * (int)sizeof(Slot3<T>) + 128;   // + slack for the 128-byte alignment
}

// resident blocks per SM the FP32 register allocation must allow
#ifndef ESI_FD3_MINB
#define ESI_FD3_MINB 3
#endif
// planes marched per loop iteration (1..4): the register queue shifts once per group
#ifndef ESI_FD3_UNROLL
#define ESI_FD3_UNROLL 4
#endif
static_assert(ESI_FD3_UNROLL >= 1 && ESI_FD3_UNROLL <= 4, "unroll 1..4");
// the centre cells of a row come from the register queue (else from shared memory)
#ifndef ESI_FD3_WQ
#define ESI_FD3_WQ 1
#endif

template <typename T, unsigned F>
__global__ void __launch_bounds__(block3<T>(), sizeof(T) == 4 ? ESI_FD3_MINB : 1) fd3_step_kernel(const __grid_constant__ StepArgs<T> a,
                                                                  int nzc) {
    constexpr int VEC = Vec3<T>::n;        // cells per consumer thread
    constexpr int NC = consumers3<T>();
    constexpr int TPR = TX3 / VEC;         // consumer threads per tile row
    extern __shared__ unsigned char smraw[];
    // TMA destinations need 128-byte alignment: align the dynamic base at run time
    Slot3<T> *ring = reinterpret_cast<Slot3<T> *>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
    // full[k]: the planes of slot k have landed; empty[k]: every consumer warp is done with them
    __shared__ __align__(8) unsigned long long full[RING3], empty[RING3];
    __shared__ double red[NC / 32];
    // per consumer warp: one value per cell of its rows (the point-source sums of a plane)
    __shared__ __align__(16) T scr_all[(F & F_PT) ? NC * VEC : 1];
    const int tid = threadIdx.x;
    const int s = blockIdx.z / nzc, zc = blockIdx.z - s * nzc;
    const int tile = ((s * nzc + zc) * a.nty + blockIdx.y) * a.ntx + blockIdx.x;
    // Receiver sampling R u_n of the input state (a.tout >= 0): the receivers whose base
    // node lies in this block's column tile and chunk, gathered from global memory by the
    // consumer threads (u_n is never written by this launch).  Point order and sums as in
    // the stand-alone gather, so the traces are the same to the bit.
    auto sample_input = [&]() {
        if (a.tout < 0 || tid >= consumers3<T>()) return;
        const T *u = a.cur + (long long)s * a.sst;
        const int r1 = a.smp.tile_ptr[tile + 1];
        for (int r = a.smp.tile_ptr[tile] + tid; r < r1; r += consumers3<T>()) {
            T v = T(0);
#pragma unroll
            for (int j = 0; j < MAXP; ++j) v += a.smp.w[r * MAXP + j] * u[a.smp.gidx[r * MAXP + j]];
            a.smp_out[a.smp.off0[r] + (long long)a.tout * a.smp.tstride[r]] = v;
        }
    };
    // Launched as a dependent of the previous step of the same loop (programmatic dependent
    // launch), everything before griddepcontrol.wait reads only what stays fixed during the
    // loop (flags, lists, sponge profiles); each thread waits for the previous step before
    // it touches a state, a field or an accumulator, and the next step may then launch.
    if (a.active && !a.active[s]) {   // a frozen shot: sampled, not stepped
        asm volatile("griddepcontrol.wait;" ::: "memory");
        sample_input();
        return;
    }
    const int x0 = blockIdx.x * TX3, y0 = blockIdx.y * TY3;
    const int zb = chunk_begin3(zc, nzc, a.nz), ze = chunk_begin3(zc + 1, nzc, a.nz);
    const int nsteps = ze - zb;
    const int J = nsteps + 2 * HALO;   // planes zb - 4 .. ze + 3 pass through the ring
    constexpr unsigned BOXU = SH3 * SW3 * sizeof(T), BOXI = TY3 * TX3 * sizeof(T);

    if (tid == 0) {
        for (int k = 0; k < RING3; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[k])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[k])),
                         "r"(NC / 32)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // plane j of the sequence is z = zb - 4 + j, in slot j % RING3; its n-th use of the slot
    // (n = j / RING3) completes phase n of full[slot], its release phase n of empty[slot]
    auto ready = [&](int j) { return mbar_wait_bounded(&full[j % RING3], (unsigned)(j / RING3) & 1u); };

    if (tid >= NC) {
        // ---- producer warp: one thread keeps the ring filled ahead of use
        if (tid != NC) return;
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        bool ok = true;
        int j = 0;
        for (; j < J; ++j) {
            if (j >= RING3 && !mbar_wait_bounded(&empty[j % RING3], (unsigned)(j / RING3 - 1) & 1u)) {
                ok = false;   // a consumer warp stopped: issue nothing more
                break;
            }
            unsigned long long *b = &full[j % RING3];
            Slot3<T> &sl = ring[j % RING3];
            const int z = zb - HALO + j;
            const bool inner = j >= HALO && j < nsteps + HALO;   // a plane this block updates
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                         "r"(inner ? BOXU + 2 * BOXI : BOXU)
                         : "memory");
            // x0 - 4 and x0 are multiples of 4 elements (16 bytes); planes outside [0, nz) read zeros
            tma_load_plane(&sl.u[0][0], &a.tm, x0 - HALO, y0 - HALO, z, s, b);
            if (inner) {
                tma_load_plane(&sl.old[0][0], &a.tm_old, x0, y0, z, s, b);
                asm volatile(
                    "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
                    " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(&sl.c[0][0])),
                    "l"(reinterpret_cast<unsigned long long>(&a.tm_cc)), "r"(x0), "r"(y0), "r"(z),
                    "r"(smem_u32(b))
                    : "memory");
            }
        }
        if (!ok) {
            atomicExch(a.dev_err, DEV_ERR_TMA_TIMEOUT);
            // let the copies in flight land before the block's shared memory is released
            for (int k = max(0, j - RING3); k < j; ++k) ready(k);
        }
        return;
    }

    // ---- consumer warps: one 16-byte row segment per thread, marching up the chunk
    const int lane = tid & 31;
    const int qx = tid % TPR, ry = tid / TPR;
    T *scr = scr_all + ((F & F_PT) ? (tid >> 5) * 32 * VEC : 0);
    (void)scr;
    const int lx = qx * VEC, gx0 = x0 + lx, gy = y0 + ry;
    const bool rowok = gy < a.ny && gx0 < a.nx;   // px >= x0 + TX3: the segment is in the pitch
    const long long plane = (long long)a.ny * a.px;
    T *po = a.po + (long long)s * a.sst;
    const long long col = (long long)gy * a.px + gx0;
    // the gather's loads overlap the producer's first TMA copies
    asm volatile("griddepcontrol.wait;" ::: "memory");
    sample_input();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    auto release = [&](int j) {   // this warp is done with plane j
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[j % RING3]))
                         : "memory");
    };
    bool late = false;
    constexpr int UN = ESI_FD3_UNROLL;
    T q[2 * HALO + UN][VEC];   // u(z - 4 .. z + 4) of the row segment, + UN - 1 planes ahead
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        late |= !ready(k);
        const Vec3<T> c = ldv3(&ring[k % RING3].u[ry + HALO][lx + HALO]);
#pragma unroll
        for (int i = 0; i < VEC; ++i) q[k][i] = c.v[i];
        // planes zb - 4 .. zb - 1 serve only their centres: free their slots at once (the
        // ring holds fewer than the 9 planes of the queue)
        if (k < HALO) release(k);
    }
    T kxy[VEC];
    bool xy_sponge = false;
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
        kxy[i] = (rowok && gx0 + i < a.nx) ? a.kx[gx0 + i] + a.ky[gy] : T(0);
        xy_sponge |= kxy[i] != T(0);
    }
    T xs = T(0), ys = T(0), zs = T(0);
    if constexpr ((F & (F_AP | F_SAD | F_CGP)) != 0) {
        xs = T(a.src_pos[3 * s + 0]);
        ys = T(a.src_pos[3 * s + 1]);
        zs = T(a.src_pos[3 * s + 2]);
    }
    (void)xs;
    (void)ys;
    (void)zs;
    int ip = 0, ie = 0;
    if constexpr ((F & F_PT) != 0) {
        ip = a.inj.tile_ptr[tile];
        ie = a.inj.tile_ptr[tile + 1];
    }
    T psum = T(0);
    const long long fbase = (long long)s * a.fst;    // caller dense fields
    const long long fb = (long long)s * a.fstp;      // internal pitched fields
    const long long dcol = (long long)gy * a.nx + gx0;
    constexpr double WK[5] = {0.0, W1, W2, W3, W4};

    // one marching step: plane z = zb + i, its z neighbours in q[O .. O + 8]
    auto plane_step = [&](auto offc, int i) {
        constexpr int O = decltype(offc)::value;
        const int z = zb + i;
        const long long gi = z * plane + col;
        const T kzz = a.kz[z];
        // the per-cell global inputs first: their latency overlaps the shared-memory loads
        // and the Laplacian below
        T ext[VEC];
        Vec3<T> r_in, p_in, ipb, app;
#pragma unroll
        for (int k = 0; k < VEC; ++k) ext[k] = r_in.v[k] = p_in.v[k] = ipb.v[k] = app.v[k] = T(0);
        if (rowok) {
            if constexpr ((F & F_EXT) != 0) {
                const T *e = a.ext + fbase + (long long)a.n * a.N + (long long)z * a.ny * a.nx + dcol;
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    if (gx0 + k < a.nx) ext[k] = e[k];
            }
            if constexpr ((F & F_CGP) != 0) {
                const long long vi = fb + (long long)a.n * a.sst + gi;
                r_in = ldv3(a.cg_r + vi);
                if (a.cg_pc > T(0)) ipb = ldv3(a.ipb2 + (long long)s * a.sst + gi);
                if (!a.cg_first) p_in = ldv3(a.cg_p + vi);
            }
            if constexpr ((F & F_AP) != 0) app = ldv3(a.ap_p + fb + (long long)a.nout * a.sst + gi);
        }
        // plane z (sequence index i + 4) has landed: the queue fill waited for it when
        // i + 4 <= 8, else the refill at the end of step i - 5; its slot is not reused
        // before this warp releases it at the end of this step
        const Slot3<T> &sl = ring[(i + HALO) % RING3];
        // point sources of this plane (entries sorted by z, then row, then column): the
        // warp scans them 32 at a time, each lane sums the entries of the warp's rows it
        // holds and leaves the sum in the owner's slot of the warp's scratch
        bool has_inj = false;
        if constexpr ((F & F_PT) != 0) {
            if (ip < ie && a.inj.cell[ip] / (TX3 * TY3) == z) {   // uniform in the warp
                has_inj = true;
#pragma unroll
                for (int k = 0; k < VEC; ++k) scr[lane * VEC + k] = T(0);
                __syncwarp();
                constexpr int RPW = 32 / TPR;   // tile rows per warp
                const int r0 = (tid >> 5) * RPW;
                int e0 = ip;
                for (;;) {
                    const int e = e0 + lane;
                    int cell = -1;
                    if (e < ie) cell = a.inj.cell[e];
                    const bool in = cell >= 0 && cell / (TX3 * TY3) == z;
                    const unsigned m = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int rem = cell - z * (TX3 * TY3);
                        const int cy = rem / TX3, cx = rem - cy * TX3;
                        if (cy >= r0 && cy < r0 + RPW) {
                            T sum = T(0);
                            for (int c = a.inj.cptr[e]; c < a.inj.cptr[e + 1]; ++c)
                                sum += a.inj.w[c] *
                                       a.inj_trace[a.inj.off0[c] + (long long)a.tin * a.inj.tstride[c]];
                            scr[((cy - r0) * TPR + cx / VEC) * VEC + cx % VEC] = sum;   // one entry per cell
                        }
                    }
                    const int cnt = __popc(m);   // the plane's entries form a prefix
                    e0 += cnt;
                    if (cnt < 32) break;
                }
                ip = e0;
                __syncwarp();
            }
        }
        if (rowok) {
            const int sy = ry + HALO;
            // x neighbours: the shared row segment [lx, lx + VEC + 8); its centre part is the
            // plane's own cells, already in the register queue
            T w[VEC + 2 * HALO];
#if ESI_FD3_WQ
#pragma unroll
            for (int c = 0; c < HALO / VEC; ++c) {
                const Vec3<T> tl = ldv3(&sl.u[sy][lx + c * VEC]);
                const Vec3<T> tr = ldv3(&sl.u[sy][lx + HALO + VEC + c * VEC]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    w[c * VEC + k] = tl.v[k];
                    w[HALO + VEC + c * VEC + k] = tr.v[k];
                }
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) w[HALO + k] = q[O + HALO][k];
#else
#pragma unroll
            for (int c = 0; c < (VEC + 2 * HALO) / VEC; ++c) {
                const Vec3<T> t = ldv3(&sl.u[sy][lx + c * VEC]);
#pragma unroll
                for (int k = 0; k < VEC; ++k) w[c * VEC + k] = t.v[k];
            }
#endif
            // Laplacian sum: 3 w0 u + sum_k w_k (6 neighbours at distance k)
            T L[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) L[k] = T(3.0 * W0) * q[O + HALO][k];
#pragma unroll
            for (int d = 1; d <= HALO; ++d) {
                const Vec3<T> up = ldv3(&sl.u[sy - d][lx + HALO]);
                const Vec3<T> dn = ldv3(&sl.u[sy + d][lx + HALO]);
#pragma unroll
                for (int k = 0; k < VEC; ++k)
                    L[k] += T(WK[d]) * (((w[k + HALO - d] + w[k + HALO + d]) + (up.v[k] + dn.v[k])) +
                                        (q[O + HALO - d][k] + q[O + HALO + d][k]));
            }
            const Vec3<T> old = ldv3(&sl.old[ry][lx]);
            const Vec3<T> cz = ldv3(&sl.c[ry][lx]);
            T src[VEC], S[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) src[k] = T(0);
            if constexpr ((F & F_EXT) != 0) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) src[k] += ext[k];
            }
            if constexpr ((F & F_CGP) != 0) {
                const long long vi = fb + (long long)a.n * a.sst + gi;
                Vec3<T> pn = r_in;
                if (a.cg_pc > T(0)) {   // z = r / (pen B^2)
#pragma unroll
                    for (int k = 0; k < VEC; ++k) pn.v[k] *= ipb.v[k];
                }
                if (!a.cg_first) {
                    const T b = T(a.cg_beta[s]);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) pn.v[k] += b * p_in.v[k];
                }
                stv3(a.cg_p + vi, pn);
#pragma unroll
                for (int k = 0; k < VEC; ++k) src[k] += pn.v[k];
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k) S[k] = L[k] + a.dx2 * src[k];
            if constexpr ((F & F_PT) != 0) {
                if (has_inj) {   // this plane's point sums, gathered by the warp
#pragma unroll
                    for (int k = 0; k < VEC; ++k) S[k] += scr[lane * VEC + k];
                }
            }
            Vec3<T> nw;
            if (xy_sponge || kzz != T(0)) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const T kap = kzz + kxy[k];
                    const T al = T(1) / (T(1) + kap);
                    const T ga = (T(1) - kap) * al;
                    const T u = q[O + HALO][k];
                    nw.v[k] = u + ga * (u - old.v[k]) + al * cz.v[k] * S[k];
                }
            } else {   // interior: alpha = gamma = 1
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const T u = q[O + HALO][k];
                    nw.v[k] = u + (u - old.v[k]) + cz.v[k] * S[k];
                }
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k)
                if (gx0 + k >= a.nx) nw.v[k] = T(0);   // pad columns stay zero
            stv3(po + gi, nw);
            if constexpr ((F & F_SAD) != 0) {
                Vec3<T> gv = ldv3(a.grad + (long long)s * a.sst + gi);
                const T ey = T(gy) * a.dx - ys, ez = T(z) * a.dx - zs;
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    const T ex = T(gx0 + k) * a.dx - xs;
                    const T B = a.unit_b ? T(1) : sqrt(ex * ex + ey * ey + ez * ez) + a.eps;
                    if (gx0 + k < a.nx) gv.v[k] += B * B * src[k] * S[k];
                }
                stv3(a.grad + (long long)s * a.sst + gi, gv);
            }
            if constexpr ((F & F_AP) != 0) {   // A p = S^T S p + pen B^2 p
                const long long vi = fb + (long long)a.nout * a.sst + gi;
                const Vec3<T> pb = ldv3(a.pb2 + (long long)s * a.sst + gi);
                Vec3<T> apv;
#pragma unroll
                for (int k = 0; k < VEC; ++k) {
                    apv.v[k] = gx0 + k < a.nx ? nw.v[k] + pb.v[k] * app.v[k] : T(0);
                    psum += app.v[k] * apv.v[k];
                }
                stv3(a.ap + vi, apv);
            }
            if constexpr ((F & F_STW) != 0) {
                Vec3<T> sv;
#pragma unroll
                for (int k = 0; k < VEC; ++k) sv.v[k] = gx0 + k < a.nx ? S[k] : T(0);
                stv3(a.stash_w + ((long long)a.slot_w * a.ns + s) * a.sst + gi, sv);
            }
            if constexpr ((F & F_GRD) != 0) {
                T *gp = a.grad + (long long)s * a.sst + gi;
                Vec3<T> gv = ldv3(gp);
                const Vec3<T> sr = ldv3(a.stash_r + ((long long)a.slot_r * a.ns + s) * a.sst + gi);
#pragma unroll
                for (int k = 0; k < VEC; ++k) gv.v[k] += nw.v[k] * sr.v[k];
                stv3(gp, gv);
            }
            if constexpr ((F & F_OUT) != 0) {
                T *o = a.fout + (long long)s * a.ofst + (long long)a.nout * a.oplane +
                       ((long long)z * a.ny + gy) * a.opx + gx0;
                if (a.opx == a.px) {   // internal pitched target: the pads get their zeros
                    stv3(o, nw);
                } else {
#pragma unroll
                    for (int k = 0; k < VEC; ++k)
                        if (gx0 + k < a.nx) o[k] = nw.v[k];
                }
            }
            if constexpr ((F & F_DFT) != 0)   // the DTFT's block stash (slot n - n0)
                stv3(a.stash_w + ((long long)a.slot_w * a.ns + s) * a.sst + gi, nw);
        }
    };
    // after step O of the group that starts at plane i: the next plane into the queue (once
    // per group the queue moves UN planes down), and release of the plane just updated
    auto refill_after = [&](auto offc, int i) {
        constexpr int O = decltype(offc)::value;
        if constexpr (O + 1 < UN) {
            if (i + O + 1 < nsteps) {   // plane z + 5 of the next step into entry O + 9
                late |= !ready(i + O + 2 * HALO + 1);
                const Vec3<T> c = ldv3(&ring[(i + O + 2 * HALO + 1) % RING3].u[ry + HALO][lx + HALO]);
#pragma unroll
                for (int e = 0; e < VEC; ++e) q[O + 2 * HALO + 1][e] = c.v[e];
            }
        } else {
            if (i + UN < nsteps) {
                late |= !ready(i + UN + 2 * HALO);
#pragma unroll
                for (int k = 0; k < 2 * HALO; ++k)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) q[k][e] = q[k + UN][e];
                const Vec3<T> c = ldv3(&ring[(i + UN + 2 * HALO) % RING3].u[ry + HALO][lx + HALO]);
#pragma unroll
                for (int e = 0; e < VEC; ++e) q[2 * HALO][e] = c.v[e];
            }
        }
        release(i + O + HALO);   // plane z: its neighbours and centre were last read in this step
    };
    for (int i = 0; i < nsteps && !__any_sync(0xffffffffu, late); i += UN) {
        plane_step(std::integral_constant<int, 0>(), i);
        refill_after(std::integral_constant<int, 0>(), i);
        if constexpr (UN >= 2) {
            if (i + 1 >= nsteps || __any_sync(0xffffffffu, late)) break;
            plane_step(std::integral_constant<int, 1>(), i + 1);
            refill_after(std::integral_constant<int, 1>(), i);
        }
        if constexpr (UN >= 3) {
            if (i + 2 >= nsteps || __any_sync(0xffffffffu, late)) break;
            plane_step(std::integral_constant<int, 2>(), i + 2);
            refill_after(std::integral_constant<int, 2>(), i);
        }
        if constexpr (UN >= 4) {
            if (i + 3 >= nsteps || __any_sync(0xffffffffu, late)) break;
            plane_step(std::integral_constant<int, 3>(), i + 3);
            refill_after(std::integral_constant<int, 3>(), i);
        }
    }
    if (late) atomicExch(a.dev_err, DEV_ERR_TMA_TIMEOUT);
    if constexpr ((F & F_AP) != 0) {
        T v = psum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[tid >> 5] = double(v);
        asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");   // consumer warps only
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NC / 32; ++w) t += red[w];
            const long long nblk = (long long)a.ntx * a.nty * nzc;
            a.dot_part[s * nblk + ((long long)zc * a.nty + blockIdx.y) * a.ntx + blockIdx.x] += t;
        }
    }
}

template <typename T, unsigned F>
cudaError_t set_smem(PerDevice &attr) {
    int set = 0;
    return per_device(attr, &set, [](int *v) {
        *v = 1;
        return cudaFuncSetAttribute(fd3_step_kernel<T, F>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, ring_bytes<T>());
    });
}

// chained: the previous launch on the stream is the previous step of the same loop, so the
// grid may be launched (programmatic dependent launch) while that step drains; its blocks
// wait for it before they read its output or write over its input.
template <typename T, unsigned F>
cudaError_t go(const StepArgs<T> &a, int ns, cudaStream_t st, bool chained) {
    const int nzc = a.ntz;
    static PerDevice attr;
    cudaError_t e = set_smem<T, F>(attr);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.ntx, a.nty, ns * nzc);
    cfg.blockDim = dim3(block3<T>());
    cfg.dynamicSmemBytes = ring_bytes<T>();
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = chained ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fd3_step_kernel<T, F>, a, nzc);
}

}  // namespace

#define ESI_CASE(FL)        \
    case (FL):              \
        return go<T, (FL)>(a, ns, st, chained);

template <typename T>
cudaError_t launch_step3(unsigned flags, const StepArgs<T> &a, int ns, cudaStream_t st,
                         bool chained) {
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
        ESI_CASE(F_EXT | F_PT | F_SAD)   // WRI: u = A^{-1}(f + q)
        ESI_CASE(F_PT | F_OUT)
        ESI_CASE(F_PT | F_AP)
        ESI_CASE(F_PT | F_GRD)
        default:
            return cudaErrorInvalidValue;
    }
}
#undef ESI_CASE

namespace {
// SMs x resident blocks per SM of the step kernel (the point-source variant stands for all:
// every FP32 variant keeps three blocks per SM, every FP64 one one)
template <typename T>
int step3_slots() {
    static PerDevice slots;
    int v = 0;
    cudaError_t e = per_device(slots, &v, [](int *out) {
        static PerDevice a2;
        cudaError_t r = set_smem<T, F_PT>(a2);
        if (r != cudaSuccess) return r;
        int dev = 0, nsm = 0, nb = 0;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
        if ((r = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return r;
        if ((r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fd3_step_kernel<T, F_PT>,
                                                               block3<T>(), ring_bytes<T>())) !=
            cudaSuccess)
            return r;
        *out = std::max(1, nb) * std::max(1, nsm);
        return cudaSuccess;
    });
    return e == cudaSuccess ? v : 1;   // unknown: the model then prefers the longest chunks
}
}  // namespace

// The chunk count that minimises (waves of resident blocks) x (planes per chunk + the
// chunk's z halo at about half the cost of a plane), with chunks of ZCH3_MIN .. ZCH3_MAX
// planes: a grid that ends in a part-filled wave leaves SMs idle at the end of every step.
int step3_chunks(int nz, long long cols, int esz) {
    const int slots = esz == 8 ? step3_slots<double>() : step3_slots<float>();
    const int lo = std::max(1, (nz + ZCH3_MAX - 1) / ZCH3_MAX);
    const int hi = std::max(lo, (nz + ZCH3_MIN - 1) / ZCH3_MIN);
    int best = lo;
    double best_cost = 1e300;
    for (int n = lo; n <= hi; ++n) {
        const long long waves = (cols * n + slots - 1) / slots;
        const double cost = (double)waves * ((double)nz / n + HALO);
        if (cost < best_cost * (1 - 1e-9)) {
            best_cost = cost;
            best = n;
        }
    }
    if (const char *ev = std::getenv("ESI_NZC3")) best = std::max(1, std::atoi(ev));
    return best;
}

template cudaError_t launch_step3<float>(unsigned, const StepArgs<float> &, int, cudaStream_t, bool);
template cudaError_t launch_step3<double>(unsigned, const StepArgs<double> &, int, cudaStream_t, bool);

}  // namespace esi
