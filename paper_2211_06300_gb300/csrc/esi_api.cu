// C-ABI entry points of libesi: context set-up (operator, sponge, geometry lists), the
// time loops of forward / adjoint modelling, the checkpointed gradient, the on-the-fly
// DTFT and Algorithm 1 (CG) on the ESI normal equation.  Host code here only enqueues
// kernels and moves a few scalars; every arithmetic step of the path runs on the GPU.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>

#include "esi_internal.h"
#include "esi_pc.h"

using namespace esi;

namespace {

// 8th-order weights at offsets 1 and 3 (Fornberg 1988).  The Nyquist symbol of the
// second difference is -4 (W1 + W3) / dx^2 per axis, which fixes the leapfrog CFL bound.
constexpr double CFL_W1 = 8.0 / 5.0, CFL_W3 = 8.0 / 315.0;

// Device allocations and graph captures are serialised over the threads of the process:
// contexts of concurrent shot groups run in threads of their own, and freeing device memory
// synchronises the device, which must not meet another thread's stream capture.
std::recursive_mutex g_dev_mu;

struct DBuf {
    void *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() {
        if (p) {
            std::lock_guard<std::recursive_mutex> lk(g_dev_mu);
            cudaFree(p);
        }
    }
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n && p) return cudaSuccess;
        std::lock_guard<std::recursive_mutex> lk(g_dev_mu);
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    template <typename U>
    U *as() const { return reinterpret_cast<U *>(p); }
};

struct HostPoint {
    std::vector<long long> node;  // global dense node index (z, y, x)
    std::vector<int> iz, iy, ix;
    std::vector<double> w;        // interpolation weight
};

struct DevInj {
    DBuf tile_ptr, cell, cptr, off0, tstride, w;
    bool empty = true;
};
struct DevSmp {
    DBuf tile_ptr, idx, gidx, w, off0, tstride, shot;
    int nrec = 0;
};

}  // namespace

struct esi_ctx {
    esi_grid g{};
    int ns = 0, nt = 0;
    double dt = 0;
    cudaStream_t st = nullptr;
    long long N = 0, sst = 0;
    int px = 0, esz = 0;
    std::vector<double> src_xyz;
    std::vector<long long> rec_off;
    std::vector<double> rec_xyz;
    double vmax = 0, vref = 0, kappa_max = 0;
    int ntx = 0, nty = 1, ntz = 0, nzc = 1, ntiles = 0;
    int dft_k = DFT_BLOCK;         // steps per blocked DTFT pass (dft_block_steps)
    DBuf cc, kz, ky, kx, src_pos;
    DBuf dev_err;                  // sticky device error word (int)
    struct TMap {
        const void *base;
        int kind;
        CUtensorMap tm;
    };
    std::vector<TMap> tmaps;       // TMA maps of state buffers and of c (by address and box)
    DevInj inj_src, inj_rec;
    DevSmp smp_rec, smp_src;
    DBuf u0, u1, a0, a1;           // forward / adjoint state pairs [ns][sst]
    DBuf part, part2, part3, scal; // reduction partials, per-shot scalars
    long long pc_fallbacks = 0;    // learned-preconditioner breakdowns (diagonal restart)
    DBuf traces;                   // scratch seismogram [nt * total receivers]
    DBuf cg_r, cg_p, cg_ap;        // CG work vectors
    DBuf pb2, ipb2;                // per-shot pen B^2 and 1 / (pen B^2) maps [ns][sst]
    PcNet *pc = nullptr;           // learned preconditioner (esi_pc_load)
    DBuf pc_img, pc_y;             // network input images (BF16) and output (FP32)
    DBuf pc_dev;                   // learned-PCG dot partials, sums and per-shot theta
    DBuf dftsnap;                  // blocked DTFT: dft_k new states [slot][ns][sst]
    DBuf wri_res;                  // WRI: data residual d - S f [traces]
    DBuf invq, invv, invpart;      // outer loop: inner solution q, model vectors, dot partials
    DBuf fdv, fdsrc, fdtr;         // frequency-domain CG: 5 complex vectors, source stash, traces
    DBuf fdsyn, fdfold, fdG;       // its twiddle tables and the Gram matrix F F^H / nt
    DBuf dsv, dseg;                // data-space CG: 5 data vectors; shot segments
    int pc_batch = 0;
    DBuf ckpt, ckpt_scale, absbits, stash, gacc, twid, dftacc;
    long long total_rec = 0;
    std::string err;
    long long launches = 0;
    // tracing: events bracketing runs of one kernel variant
    struct Pending {
        std::string name;
        double bpc;
        long long launches, cells;
        cudaEvent_t a, b;
    };
    struct Stat {
        std::string name;
        double bpc = 0;
        long long launches = 0, cells = 0;
        double ms = 0;
    };
    bool prof = false;
    int prof_active = 0;  // shots being advanced (cells per launch = prof_active * N)
    // CUDA graphs of whole time loops, keyed by the loop's launch parameters.  Captured on a
    // private stream (capture is not allowed on the legacy default stream) and launched on
    // the context stream; replays of an identical loop skip the per-step launch cost.
    struct GraphEntry {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec;
        long long kernels;
        unsigned long long used;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap = nullptr;
    bool use_graphs = true;
    bool pdl = true;               // loop steps after the first start as dependent launches
    unsigned long long graph_clock = 0;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> evpool;
    std::vector<Stat> stats;
    // concurrent shot groups (esi_set_shot_groups): child contexts over contiguous shot
    // ranges, each on a stream of its own; the batch calls fan out to them
    std::vector<esi_ctx *> grp;
    std::vector<int> grp_s0;           // first shot of each group, then ns
    std::vector<cudaStream_t> grp_st;
    std::vector<cudaEvent_t> grp_ev;   // [0] fork, [1 + g] join of group g
    DBuf grp_grad;                     // the groups' partial gradients [G][N]

    void clear_groups() {
        for (auto *c : grp) esi_destroy(c);
        for (auto st : grp_st) cudaStreamDestroy(st);
        for (auto ev : grp_ev) cudaEventDestroy(ev);
        grp.clear();
        grp_s0.clear();
        grp_st.clear();
        grp_ev.clear();
    }

    ~esi_ctx() {
        clear_groups();
        if (pc) pcnet_destroy(pc);
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        if (cap) cudaStreamDestroy(cap);
        for (auto &p : pending) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        for (auto e : evpool) cudaEventDestroy(e);
    }

    esi_status fail(esi_status s, const std::string &m) {
        err = m;
        return s;
    }
};

#define CK(expr)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return ctx->fail(_e == cudaErrorMemoryAllocation ? ESI_ERR_OOM : ESI_ERR_CUDA,  \
                             std::string(#expr) + ": " + cudaGetErrorString(_e));         \
    } while (0)

#define CKL(expr)        \
    do {                 \
        CK(expr);        \
        ++ctx->launches; \
    } while (0)

namespace {

cudaEvent_t prof_mark(esi_ctx *ctx) {
    if (!ctx->prof) return nullptr;
    cudaEvent_t e = nullptr;
    if (!ctx->evpool.empty()) {
        e = ctx->evpool.back();
        ctx->evpool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, ctx->st);
    return e;
}

void prof_close(esi_ctx *ctx, cudaEvent_t a, const std::string &name, double bpc,
                long long launches, long long cells) {
    if (!a) return;
    cudaEvent_t b = prof_mark(ctx);
    if (!b) {
        ctx->evpool.push_back(a);
        return;
    }
    ctx->pending.push_back({name, bpc, launches, cells, a, b});
}

std::string step_name(const esi_ctx *ctx, unsigned f) {
    static const char *names[] = {"EXT", "CGP", "PT", "SMP", "OUT", "AP", "STW", "GRD", "SAD", "DFT"};
    std::string s = ctx->g.ndim == 2 ? "fd2_step[" : "fd3_step[";
    bool first = true;
    for (int i = 0; i < 10; ++i)
        if (f & (1u << i)) {
            if (!first) s += "|";
            s += names[i];
            first = false;
        }
    return s + "]";
}

// algorithmic HBM bytes per cell update of a step variant: the stencil reads u_n, u_{n-1}
// and c and writes u_{n+1}; each fused stream adds its own reads / writes.  The CG forward
// half reads r and p and writes p (+ the 1/(beta B^2) map under a preconditioner, + a
// quarter float of the learned correction); the CG product epilogue reads p and the
// beta B^2 map and writes A p.
double step_bpc(const esi_ctx *ctx, unsigned f, int nf, bool pc = false, bool learned = false) {
    const double e = ctx->esz;
    double b = 4 * e;
    if (f & F_EXT) b += e;
    if (f & F_CGP) b += 3 * e + (pc ? e : 0.0) + (learned ? 1.0 : 0.0);
    if (f & F_OUT) b += e;
    if (f & F_AP) b += 3 * e;
    if (f & F_STW) b += e;
    if (f & F_GRD) b += 3 * e;
    if (f & F_SAD) b += 2 * e;
    if (f & F_DFT) b += e;   // the state into the DTFT block stash
    return b;
}

template <typename U>
cudaError_t upload(DBuf &b, const std::vector<U> &v, cudaStream_t st) {
    cudaError_t e = b.ensure(std::max<size_t>(v.size() * sizeof(U), 16));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, st);
}

// bilinear / trilinear weights of a point; nodes in z-major order; zero weights dropped
bool point_weights(const esi_grid &g, const double *xyz, HostPoint &hp, int &iz0, int &iy0,
                   int &ix0) {
    hp = HostPoint();
    double pos[3] = {xyz[2], xyz[1], xyz[0]};  // (z, y, x)
    int n[3] = {g.nz, g.ny, g.nx};
    int base[3] = {0, 0, 0};
    std::vector<std::pair<int, double>> ax[3];
    for (int a = 0; a < 3; ++a) {
        if (a == 1 && g.ndim == 2) {
            ax[a].push_back({0, 1.0});
            continue;
        }
        const double f = pos[a] / g.dx;
        const double fl = std::floor(f);
        const int i0 = (int)fl;
        const double w1 = f - fl;
        base[a] = i0;
        if (1.0 - w1 != 0.0) ax[a].push_back({i0, 1.0 - w1});
        if (w1 != 0.0) ax[a].push_back({i0 + 1, w1});
        for (auto &pw : ax[a])
            if (pw.first < 0 || pw.first >= n[a]) return false;
    }
    iz0 = base[0];
    iy0 = base[1];
    ix0 = base[2];
    for (auto &pz : ax[0])
        for (auto &py : ax[1])
            for (auto &pxw : ax[2]) {
                hp.iz.push_back(pz.first);
                hp.iy.push_back(py.first);
                hp.ix.push_back(pxw.first);
                hp.node.push_back(((long long)pz.first * g.ny + py.first) * g.nx + pxw.first);
                hp.w.push_back(pz.second * py.second * pxw.second);
            }
    return true;
}

struct Contrib {
    long long off0;
    int tstride;
    double w;
};

// tile index and local cell of a node for the step kernels
void tile_of(const esi_ctx *c, int s, int iz, int iy, int ix, int &tile, int &cell) {
    if (c->g.ndim == 2) {
        const int bz = iz / TZ2, bx = ix / TX2;
        tile = (s * c->ntz + bz) * c->ntx + bx;
        cell = (iz - bz * TZ2) * TX2 + (ix - bx * TX2);
    } else {
        int zc = 0;
        while (zc + 1 < c->nzc && chunk_begin3(zc + 1, c->nzc, c->g.nz) <= iz) ++zc;
        const int by = iy / TY3, bx = ix / TX3;
        tile = ((s * c->nzc + zc) * c->nty + by) * c->ntx + bx;
        cell = iz * (TX3 * TY3) + (iy - by * TY3) * TX3 + (ix - bx * TX3);
    }
}

template <typename T>
esi_status build_inj(esi_ctx *ctx, DevInj &out,
                     const std::vector<std::vector<std::pair<HostPoint, Contrib>>> &per_shot) {
    // per (tile) -> ordered map cell -> contributions
    const int ntt = ctx->ns * ctx->ntiles;
    std::vector<std::map<int, std::vector<Contrib>>> tiles(ntt);
    for (int s = 0; s < ctx->ns; ++s)
        for (auto &pc : per_shot[s]) {
            const HostPoint &hp = pc.first;
            for (size_t k = 0; k < hp.node.size(); ++k) {
                int tile, cell;
                tile_of(ctx, s, hp.iz[k], hp.iy[k], hp.ix[k], tile, cell);
                Contrib c = pc.second;
                c.w *= hp.w[k];
                tiles[tile][cell].push_back(c);
            }
        }
    std::vector<int> tile_ptr(ntt + 1, 0), cell, cptr(1, 0), tstr;
    std::vector<long long> off0;
    std::vector<T> w;
    for (int t = 0; t < ntt; ++t) {
        for (auto &kv : tiles[t]) {  // std::map: cells ascending (z-sorted in 3D)
            cell.push_back(kv.first);
            for (auto &c : kv.second) {
                off0.push_back(c.off0);
                tstr.push_back(c.tstride);
                w.push_back(T(c.w));
            }
            cptr.push_back((int)off0.size());
        }
        tile_ptr[t + 1] = (int)cell.size();
    }
    out.empty = cell.empty();
    CK(upload(out.tile_ptr, tile_ptr, ctx->st));
    CK(upload(out.cell, cell, ctx->st));
    CK(upload(out.cptr, cptr, ctx->st));
    CK(upload(out.off0, off0, ctx->st));
    CK(upload(out.tstride, tstr, ctx->st));
    CK(upload(out.w, w, ctx->st));
    return ESI_OK;
}

struct SmpHost {
    int s;
    HostPoint hp;
    int iz0, iy0, ix0;
    long long off0;
    int tstride;
    double scale;
};

template <typename T>
esi_status build_smp(esi_ctx *ctx, DevSmp &out, const std::vector<SmpHost> &recs) {
    const int ntt = ctx->ns * ctx->ntiles;
    std::vector<std::vector<int>> by_tile(ntt);
    for (size_t r = 0; r < recs.size(); ++r) {
        int tile, cell;
        tile_of(ctx, recs[r].s, recs[r].iz0, recs[r].iy0, recs[r].ix0, tile, cell);
        by_tile[tile].push_back((int)r);
    }
    std::vector<int> tile_ptr(ntt + 1, 0), idx, tstr, shot;
    std::vector<long long> gidx, off0;
    std::vector<T> w;
    for (int t = 0; t < ntt; ++t) {
        for (int r : by_tile[t]) {
            const SmpHost &h = recs[r];
            const int lz0 = h.iz0 % TZ2, lx0 = h.ix0 % TX2;
            const long long gbase = ((long long)h.iz0 * ctx->g.ny + h.iy0) * ctx->px + h.ix0;
            const int sbase = (lz0 + HALO) * SW2 + (lx0 + HALO);
            for (int j = 0; j < MAXP; ++j) {
                if (j < (int)h.hp.node.size()) {
                    const int dz = h.hp.iz[j] - h.iz0, dy = h.hp.iy[j] - h.iy0, dxx = h.hp.ix[j] - h.ix0;
                    idx.push_back(sbase + dz * SW2 + dxx);
                    gidx.push_back(((long long)h.hp.iz[j] * ctx->g.ny + h.hp.iy[j]) * ctx->px +
                                   h.hp.ix[j]);
                    (void)dy;
                    w.push_back(T(h.hp.w[j] * h.scale));
                } else {
                    idx.push_back(sbase);
                    gidx.push_back(gbase);
                    w.push_back(T(0));
                }
            }
            off0.push_back(h.off0);
            tstr.push_back(h.tstride);
            shot.push_back(h.s);
        }
        tile_ptr[t + 1] = (int)off0.size();
    }
    // 2D in-kernel sampling uses 4 points in (z0,x0),(z0,x1),(z1,x0),(z1,x1) order; the
    // host lists hold only the nonzero ones in that order, padded with zero weights, so
    // the sum order matches the node order of the definition.
    out.nrec = (int)off0.size();
    CK(upload(out.tile_ptr, tile_ptr, ctx->st));
    CK(upload(out.idx, idx, ctx->st));
    CK(upload(out.gidx, gidx, ctx->st));
    CK(upload(out.w, w, ctx->st));
    CK(upload(out.off0, off0, ctx->st));
    CK(upload(out.tstride, tstr, ctx->st));
    CK(upload(out.shot, shot, ctx->st));
    return ESI_OK;
}

template <typename T>
InjList<T> inj_view(const DevInj &d) {
    InjList<T> l;
    l.tile_ptr = d.tile_ptr.as<int>();
    l.cell = d.cell.as<int>();
    l.cptr = d.cptr.as<int>();
    l.off0 = d.off0.as<long long>();
    l.tstride = d.tstride.as<int>();
    l.w = d.w.as<T>();
    return l;
}

template <typename T>
SmpList<T> smp_view(const DevSmp &d) {
    SmpList<T> l;
    l.tile_ptr = d.tile_ptr.as<int>();
    l.idx = d.idx.as<int>();
    l.gidx = d.gidx.as<long long>();
    l.w = d.w.as<T>();
    l.off0 = d.off0.as<long long>();
    l.tstride = d.tstride.as<int>();
    l.shot = d.shot.as<int>();
    l.nrec = d.nrec;
    return l;
}

}  // namespace

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
TensorMapEncoder esi::tensor_map_encoder() {
    static TensorMapEncoder fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncoder>(p);
    });
    return fn;
}

namespace {

// TMA maps (cells outside the grid are zero-filled by the copy engine):
//   kind 0, a state buffer with the halo box: 2D [ns][nz][px] as dims (nx, nz, ns), box
//     (SW2, SH2, 1); 3D [ns][nz][ny][px] as dims (nx, ny, nz, ns), box (SW3, SH3, 1, 1);
//   kind 1, a 3D state buffer with the tile-interior box (TX3, TY3, 1, 1);
//   kind 2, the 3D array c [nz][ny][px] as dims (nx, ny, nz), box (TX3, TY3, 1);
//   2D tile-interior boxes (TX2, TZ2) of the CG-product streams: kind 3, a per-shot array
//   [ns][nz][px] (states, lambda B^2 maps); kind 4, c [nz][px]; kind 5, a space-time vector
//   [ns][nt][nz][px] as dims (nx, nz, nt, ns).
bool state_map(esi_ctx *ctx, const void *base, CUtensorMap *out, int kind = 0) {
    for (auto &m : ctx->tmaps)
        if (m.base == base && m.kind == kind) {
            *out = m.tm;
            return true;
        }
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    CUtensorMap tm;
    const cuuint64_t row = (cuuint64_t)ctx->px * ctx->esz, shot = (cuuint64_t)ctx->sst * ctx->esz;
    const cuuint64_t nx = ctx->g.nx, ny = ctx->g.ny, nz = ctx->g.nz, ns = ctx->ns;
    cuuint64_t dims[4];
    cuuint64_t str[3];
    cuuint32_t box[4];
    cuuint32_t rank;
    if (ctx->g.ndim == 2) {
        rank = 3;
        dims[0] = nx, dims[1] = nz, dims[2] = ns;
        str[0] = row, str[1] = shot;
        box[0] = SW2, box[1] = SH2, box[2] = 1;
    } else if (kind == 2) {
        rank = 3;
        dims[0] = nx, dims[1] = ny, dims[2] = nz;
        str[0] = row, str[1] = row * ny;
        box[0] = TX3, box[1] = TY3, box[2] = 1;
    } else {
        rank = 4;
        dims[0] = nx, dims[1] = ny, dims[2] = nz, dims[3] = ns;
        str[0] = row, str[1] = row * ny, str[2] = shot;
        box[0] = kind == 1 ? TX3 : SW3, box[1] = kind == 1 ? TY3 : SH3, box[2] = 1, box[3] = 1;
    }
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&tm, ctx->esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     rank, const_cast<void *>(base), dims, str, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    ctx->tmaps.push_back({base, kind, tm});
    *out = tm;
    return true;
}

template <typename T>
StepArgs<T> base_args(esi_ctx *ctx) {
    StepArgs<T> a;
    std::memset(&a, 0, sizeof(a));
    a.nz = ctx->g.nz;
    a.ny = ctx->g.ny;
    a.nx = ctx->g.nx;
    a.px = ctx->px;
    a.sst = ctx->sst;
    a.N = ctx->N;
    a.fst = ctx->N * ctx->nt;
    a.fstp = ctx->sst * ctx->nt;
    a.ntx = ctx->ntx;
    a.nty = ctx->nty;
    a.ntz = ctx->ntz;
    a.cc = ctx->cc.as<T>();
    a.kz = ctx->kz.as<T>();
    a.ky = ctx->ky.as<T>();
    a.kx = ctx->kx.as<T>();
    a.dx2 = T(ctx->g.dx * ctx->g.dx);
    a.dx = T(ctx->g.dx);
    a.src_pos = ctx->src_pos.as<double>();
    a.ns = ctx->ns;
    a.tout = -1;
    a.dev_err = ctx->dev_err.as<int>();
    return a;
}

// One step of either kernel.  In 3D the step kernel samples its input state itself when
// F_SMP is set (a.tout >= 0), by a gather of the receivers of each block's tile.
template <typename T>
esi_status step(esi_ctx *ctx, unsigned flags, const StepArgs<T> &a, bool chained = false) {
    StepArgs<T> b = a;
    if (!state_map(ctx, a.cur, &b.tm) ||
        (ctx->g.ndim == 3 && (!state_map(ctx, a.po, &b.tm_old, 1) || !state_map(ctx, a.cc, &b.tm_cc, 2))))
        return ctx->fail(ESI_ERR_CUDA, "cuTensorMapEncodeTiled failed for a state buffer");
    if (ctx->g.ndim == 2) {
        CKL(launch_step2<T>(flags, b, ctx->ns, ctx->st, chained && ctx->pdl));
    } else {
        if (!(flags & F_SMP) || a.smp.nrec == 0) b.tout = -1;
        CKL(launch_step3<T>(flags & ~F_SMP, b, ctx->ns, ctx->st, chained && ctx->pdl));
    }
    return ESI_OK;
}

template <typename T>
esi_status setup_model(esi_ctx *ctx, const void *vel, bool first) {
    const int nblk = 1024;
    CK(ctx->part.ensure(sizeof(double) * std::max<long long>(nblk, 1)));
    CK(cudaMemsetAsync(ctx->cc.p, 0, ctx->sst * sizeof(T), ctx->st));
    CKL(launch_setup_cc<T>(reinterpret_cast<const T *>(vel), ctx->cc.as<T>(), ctx->g.nz, ctx->g.ny,
                           ctx->g.nx, ctx->px, ctx->dt, ctx->g.dx, ctx->part.as<double>(), nblk,
                           ctx->st));
    std::vector<double> vm(nblk);
    CK(cudaMemcpyAsync(vm.data(), ctx->part.p, nblk * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    double vmax = 0;
    for (double v : vm) vmax = std::max(vmax, v);
    if (!(vmax > 0) || !std::isfinite(vmax))
        return ctx->fail(ESI_ERR_ARG, "velocity must be positive and finite");
    const double limit = std::sqrt(1.0 / (ctx->g.ndim * (CFL_W1 + CFL_W3)));
    if (vmax * ctx->dt / ctx->g.dx > limit)
        return ctx->fail(ESI_ERR_CFL, "v_max dt / dx = " + std::to_string(vmax * ctx->dt / ctx->g.dx) +
                                          " exceeds the stability limit " + std::to_string(limit));
    ctx->vmax = vmax;
    if (first) {
        ctx->vref = ctx->g.sponge_vref > 0 ? ctx->g.sponge_vref : vmax;
        // sponge: kappa = eta dt / 2, eta = eta_max sum_axes (d / nb)^2,
        // eta_max = 3 vref ln(1/R) / (2 nb dx)
        const int nb = ctx->g.nb;
        const double eta_max =
            nb > 0 ? 3.0 * ctx->vref * std::log(1.0 / ctx->g.sponge_R) / (2.0 * nb * ctx->g.dx) : 0.0;
        ctx->kappa_max = eta_max * ctx->dt / 2.0;
        auto prof = [&](int n, bool used, int len) {
            std::vector<T> p(std::max(len, 1), T(0));
            if (!used || nb <= 0) return p;
            for (int i = 0; i < n; ++i) {
                const int d = std::max(std::max(nb - i, i - (n - 1 - nb)), 0);
                const double r = double(d) / nb;
                p[i] = T(ctx->kappa_max * r * r);
            }
            return p;
        };
        CK(upload(ctx->kz, prof(ctx->g.nz, true, ctx->g.nz), ctx->st));
        CK(upload(ctx->ky, prof(ctx->g.ny, ctx->g.ndim == 3, ctx->g.ny), ctx->st));
        // padded to the x pitch (zeros) for 16-byte loads
        CK(upload(ctx->kx, prof(ctx->g.nx, true, ctx->px), ctx->st));
    }
    return ESI_OK;
}

template <typename T>
esi_status setup_geometry(esi_ctx *ctx) {
    const esi_grid &g = ctx->g;
    const int d = g.ndim;
    std::vector<std::vector<std::pair<HostPoint, Contrib>>> src_inj(ctx->ns), rec_inj(ctx->ns);
    std::vector<SmpHost> rec_smp, src_smp;
    for (int s = 0; s < ctx->ns; ++s) {
        HostPoint hp;
        int iz0, iy0, ix0;
        if (!point_weights(g, &ctx->src_xyz[3 * s], hp, iz0, iy0, ix0))
            return ctx->fail(ESI_ERR_ARG, "source " + std::to_string(s) + " outside the grid");
        // forward injection carries f_n w / dx^d; the kernel adds dx^2 * q
        src_inj[s].push_back({hp, Contrib{(long long)s * ctx->nt, 1, std::pow(g.dx, 2 - d)}});
        src_smp.push_back(SmpHost{s, hp, iz0, iy0, ix0, (long long)s * ctx->nt, 1, std::pow(g.dx, -d)});
        const int nr = (int)(ctx->rec_off[s + 1] - ctx->rec_off[s]);
        for (int r = 0; r < nr; ++r) {
            const double *xyz = &ctx->rec_xyz[3 * (ctx->rec_off[s] + r)];
            if (!point_weights(g, xyz, hp, iz0, iy0, ix0))
                return ctx->fail(ESI_ERR_ARG, "receiver " + std::to_string(r) + " of shot " +
                                                  std::to_string(s) + " outside the grid");
            const long long off0 = (long long)ctx->nt * ctx->rec_off[s] + r;
            rec_inj[s].push_back({hp, Contrib{off0, nr, g.dx * g.dx}});
            rec_smp.push_back(SmpHost{s, hp, iz0, iy0, ix0, off0, nr, 1.0});
        }
    }
    esi_status e;
    if ((e = build_inj<T>(ctx, ctx->inj_src, src_inj)) != ESI_OK) return e;
    if ((e = build_inj<T>(ctx, ctx->inj_rec, rec_inj)) != ESI_OK) return e;
    if ((e = build_smp<T>(ctx, ctx->smp_rec, rec_smp)) != ESI_OK) return e;
    if ((e = build_smp<T>(ctx, ctx->smp_src, src_smp)) != ESI_OK) return e;
    CK(upload(ctx->src_pos, ctx->src_xyz, ctx->st));
    return ESI_OK;
}

template <typename T>
esi_status ensure_states(esi_ctx *ctx, bool adj) {
    const size_t b = (size_t)ctx->ns * ctx->sst * sizeof(T);
    CK(ctx->u0.ensure(b));
    CK(ctx->u1.ensure(b));
    if (adj) {
        CK(ctx->a0.ensure(b));
        CK(ctx->a1.ensure(b));
    }
    return ESI_OK;
}

// Reads the sticky device error word (after a synchronisation point of the call).
esi_status check_dev_err(esi_ctx *ctx) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, ctx->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (h == DEV_ERR_TMA_TIMEOUT)
        return ctx->fail(ESI_ERR_TIMEOUT, "a TMA tile wait ran out of its iteration limit");
    if (h) return ctx->fail(ESI_ERR_TIMEOUT, "device error word " + std::to_string(h));
    return ESI_OK;
}

// ------------------------------------------------------------------ loop graphs
constexpr int GRAPH_MIN_STEPS = 32;   // shorter loops are launched directly
constexpr size_t GRAPH_CACHE = 8;      // instantiated loops kept per context

template <typename T>
std::vector<unsigned char> loop_key(const StepArgs<T> &a, unsigned flags, int dir, int i0, int i1,
                                    bool sample_src, const T *cur, const T *po) {
    std::vector<unsigned char> k(sizeof(a) + 64);
    std::memcpy(k.data(), &a, sizeof(a));  // base_args zero-fills, so padding is zero
    unsigned char *q = k.data() + sizeof(a);
    std::memset(q, 0, 64);
    std::memcpy(q, &flags, 4);
    std::memcpy(q + 4, &dir, 4);
    std::memcpy(q + 8, &i0, 4);
    std::memcpy(q + 12, &i1, 4);
    const int ss = sample_src;
    std::memcpy(q + 16, &ss, 4);
    std::memcpy(q + 24, &cur, sizeof(cur));
    std::memcpy(q + 32, &po, sizeof(po));
    return k;
}

// Launch a cached graph of this loop if present; returns true when it did.
bool graph_replay(esi_ctx *ctx, const std::vector<unsigned char> &key, esi_status &st) {
    for (auto &g : ctx->graphs)
        if (g.key == key) {
            cudaError_t e = cudaGraphLaunch(g.exec, ctx->st);
            if (e != cudaSuccess) {
                st = ctx->fail(ESI_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
            } else {
                st = ESI_OK;
                ctx->launches += g.kernels;
                g.used = ++ctx->graph_clock;
            }
            return true;
        }
    return false;
}

// Capture `body` (which enqueues on ctx->st) into a graph, cache it and launch it.
template <typename F>
esi_status graph_capture(esi_ctx *ctx, std::vector<unsigned char> &&key, F &&body) {
    if (!ctx->cap) CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    std::lock_guard<std::recursive_mutex> lk(g_dev_mu);   // no allocation meets the capture
    cudaStream_t user = ctx->st;
    const long long l0 = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    ctx->st = ctx->cap;
    esi_status e = body();
    ctx->st = user;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != ESI_OK) {
        if (graph) cudaGraphDestroy(graph);
        return e;
    }
    if (ce != cudaSuccess) return ctx->fail(ESI_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess)
        return ctx->fail(ESI_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
    const long long kernels = ctx->launches - l0;
    ctx->launches = l0;  // counted when the graph runs
    if (ctx->graphs.size() >= GRAPH_CACHE) {
        auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](const esi_ctx::GraphEntry &x, const esi_ctx::GraphEntry &y) {
                                        return x.used < y.used;
                                    });
        cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
    }
    ctx->graphs.push_back({std::move(key), exec, kernels, ++ctx->graph_clock});
    esi_status st;
    graph_replay(ctx, ctx->graphs.back().key, st);
    return st;
}

// ------------------------------------------------------------------ forward modelling
// Runs steps [n0, n1) starting from states (cur, po) = (u_{n0}, u_{n0-1}); on return
// cur holds u_{n1}.  Sampling of the inputs writes traces[n-1].
template <typename T>
esi_status fwd_loop(esi_ctx *ctx, StepArgs<T> a, unsigned flags, T *&cur, T *&po, int n0,
                    int n1, std::vector<std::pair<int, int>> *ckpt_at = nullptr) {
    (void)ckpt_at;
    cudaEvent_t ev = prof_mark(ctx);
    T *c0 = cur, *p0 = po;
    auto body = [&]() -> esi_status {
        T *c = c0, *q = p0;
        for (int n = n0; n < n1; ++n) {
            a.cur = c;
            a.po = q;
            a.n = n;
            a.tin = n;
            a.tout = n - 1;
            a.slot_w = n - n0;
            esi_status e = step<T>(ctx, flags, a, n > n0);
            if (e != ESI_OK) return e;
            std::swap(c, q);
        }
        return ESI_OK;
    };
    esi_status e;
    if (ctx->use_graphs && n1 - n0 >= GRAPH_MIN_STEPS) {
        auto key = loop_key(a, flags, +1, n0, n1, false, c0, p0);
        if (!graph_replay(ctx, key, e)) e = graph_capture(ctx, std::move(key), body);
    } else {
        e = body();
    }
    if (e != ESI_OK) return e;
    if ((n1 - n0) & 1) std::swap(cur, po);
    prof_close(ctx, ev, step_name(ctx, flags),
               step_bpc(ctx, flags, a.nf, a.cg_pc > T(0), a.pc_y != nullptr), n1 - n0,
               (long long)(n1 - n0) * ctx->prof_active * ctx->N);
    return ESI_OK;
}

// Forward modelling with the blocked DTFT: steps [n0, n0 + K) store their new states in the
// stash, then one launch folds them into the accumulators; the whole run is one graph.
template <typename T>
esi_status fwd_dft_loop(esi_ctx *ctx, StepArgs<T> a, unsigned flags, T *cur, T *po, T *tr) {
    cudaEvent_t ev = prof_mark(ctx);
    const int nt = ctx->nt;
    auto body = [&]() -> esi_status {
        T *c = cur, *q = po;
        for (int n0 = 0; n0 < nt; n0 += ctx->dft_k) {
            const int n1 = std::min(nt, n0 + ctx->dft_k);
            for (int n = n0; n < n1; ++n) {
                a.cur = c;
                a.po = q;
                a.n = n;
                a.tin = n;
                a.tout = n - 1;
                a.slot_w = n - n0;
                esi_status e = step<T>(ctx, flags, a, n > 0);
                if (e != ESI_OK) return e;
                std::swap(c, q);
            }
            CKL(launch_dft_block<T>(a.stash_w, n1 - n0, ctx->ns, ctx->sst, ctx->g.nx, ctx->px, a.nf,
                                    a.twid + (size_t)n0 * a.nf * 2, a.dft, ctx->st));
        }
        CKL(launch_sample_global<T>(a.smp, c, ctx->sst, tr, nt - 1, ctx->st));
        return ESI_OK;
    };
    esi_status e;
    if (ctx->use_graphs && nt >= GRAPH_MIN_STEPS) {
        auto key = loop_key(a, flags, +2, 0, nt, false, cur, po);
        if (!graph_replay(ctx, key, e)) e = graph_capture(ctx, std::move(key), body);
    } else {
        e = body();
    }
    if (e != ESI_OK) return e;
    // the stencil and the stash store per step, plus the block pass: the stash once more
    // and the accumulators' read and write once per block
    const double es = double(sizeof(T));
    prof_close(ctx, ev, step_name(ctx, flags) + "+dft_block",
               step_bpc(ctx, flags, a.nf) + es + 4.0 * a.nf * es / ctx->dft_k, nt + (nt + ctx->dft_k - 1) / ctx->dft_k,
               (long long)nt * ctx->prof_active * ctx->N);
    return ESI_OK;
}

template <typename T>
esi_status forward_impl(esi_ctx *ctx, const void *wavelet, const void *ext, void *traces,
                        const double *freqs, int nf, T *dft_acc) {
    ctx->prof_active = ctx->ns;
    esi_status e = ensure_states<T>(ctx, false);
    if (e != ESI_OK) return e;
    CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
    CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
    StepArgs<T> a = base_args<T>(ctx);
    unsigned flags = F_SMP;
    if (wavelet) {
        flags |= F_PT;
        a.inj = inj_view<T>(ctx->inj_src);
        a.inj_trace = reinterpret_cast<const T *>(wavelet);
    }
    if (ext) {
        flags |= F_EXT;
        a.ext = reinterpret_cast<const T *>(ext);
    }
    if (!wavelet && !ext) return ctx->fail(ESI_ERR_ARG, "no source given");
    a.smp = smp_view<T>(ctx->smp_rec);
    T *tr = reinterpret_cast<T *>(traces);
    if (!tr) {
        CK(ctx->traces.ensure(std::max<size_t>((size_t)ctx->total_rec * ctx->nt * sizeof(T), 16)));
        tr = ctx->traces.as<T>();
    }
    a.smp_out = tr;
    T *cur = ctx->u0.as<T>(), *po = ctx->u1.as<T>();
    if (nf > 0) {
        // blocked DTFT: each step stores u_{n+1} in a dft_k-slot stash, and one pass per
        // block adds the block's terms to the accumulators (80 -> 8 + 80 / dft_k bytes per
        // cell update for five frequencies)
        flags |= F_DFT;
        std::vector<T> tw((size_t)ctx->nt * nf * 2);
        for (int n = 0; n < ctx->nt; ++n)
            for (int m = 0; m < nf; ++m) {
                const double ph = 2.0 * M_PI * freqs[m] * (n + 1) * ctx->dt;
                tw[((size_t)n * nf + m) * 2] = T(std::cos(ph));
                tw[((size_t)n * nf + m) * 2 + 1] = T(std::sin(ph));
            }
        CK(upload(ctx->twid, tw, ctx->st));
        CK(ctx->dftsnap.ensure((size_t)ctx->dft_k * ctx->ns * ctx->sst * sizeof(T)));
        a.nf = nf;
        a.twid = ctx->twid.as<T>();
        a.dft = dft_acc;
        a.stash_w = ctx->dftsnap.as<T>();
        return fwd_dft_loop<T>(ctx, a, flags, cur, po, tr);
    }
    e = fwd_loop<T>(ctx, a, flags, cur, po, 0, ctx->nt);
    if (e != ESI_OK) return e;
    CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, tr, ctx->nt - 1, ctx->st));
    return ESI_OK;
}

// ------------------------------------------------------------------ allocation-free forward
// Scratch of esi_forward_noalloc: the two wave states live in this file-scope device array
// instead of context-owned cudaMalloc buffers.  Every GPU that loads the library holds it
// until the process exits.  Host code must not use the symbol as an address (on the host
// it names a stand-in); the device address is fetched once per device below.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128] = {nullptr};

// Device address of the scratch array for the current device (set-up on first use).
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

template <typename T>
esi_status forward_noalloc_impl(esi_ctx *ctx, const void *wavelet, const void *ext, void *traces) {
    if (!wavelet && !ext) return ctx->fail(ESI_ERR_ARG, "no source given");
    const size_t need = 2 * (size_t)ctx->ns * ctx->sst * sizeof(T);
    if (need > NOALLOC_SCRATCH_BYTES)
        return ctx->fail(ESI_ERR_ARG, "esi_forward_noalloc: the two wave states need " +
                                          std::to_string(need) + " bytes, above the " +
                                          std::to_string(NOALLOC_SCRATCH_BYTES) +
                                          "-byte static scratch; use esi_forward");
    void *base = nullptr;
    CK(noalloc_scratch(&base));
    // the array keeps the previous call's contents: both states must start at zero
    CK(cudaMemsetAsync(base, 0, need, ctx->st));
    T *cur = reinterpret_cast<T *>(base);
    T *po = cur + (size_t)ctx->ns * ctx->sst;
    StepArgs<T> a = base_args<T>(ctx);
    unsigned flags = F_SMP;
    if (wavelet) {
        flags |= F_PT;
        a.inj = inj_view<T>(ctx->inj_src);
        a.inj_trace = reinterpret_cast<const T *>(wavelet);
    }
    if (ext) {
        flags |= F_EXT;
        a.ext = reinterpret_cast<const T *>(ext);
    }
    a.smp = smp_view<T>(ctx->smp_rec);
    a.smp_out = reinterpret_cast<T *>(traces);
    // the same launches as esi_forward's loop, without its graph cache (instantiating a
    // CUDA graph may take device memory): every step after the first is a programmatic
    // dependent launch, and the run is timed for esi_get_profile like the other loops
    ctx->prof_active = ctx->ns;
    cudaEvent_t ev = prof_mark(ctx);
    for (int n = 0; n < ctx->nt; ++n) {
        a.cur = cur;
        a.po = po;
        a.n = n;
        a.tin = n;
        a.tout = n - 1;
        esi_status e = step<T>(ctx, flags, a, n > 0);
        if (e != ESI_OK) return e;
        std::swap(cur, po);
    }
    prof_close(ctx, ev, step_name(ctx, flags), step_bpc(ctx, flags, a.nf), ctx->nt,
               (long long)ctx->nt * ctx->prof_active * ctx->N);
    CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, a.smp_out, ctx->nt - 1, ctx->st));
    return ESI_OK;
}

// ------------------------------------------------------------------ adjoint modelling
// Time-reversed run: for j = j1 .. j0+1 computes lambda_j from (lambda_{j+1}, lambda_{j+2})
// with source R^T e_{j-1}.  Epilogue writes index j-1 of the dense outputs.
template <typename T>
esi_status adj_loop(esi_ctx *ctx, StepArgs<T> a, unsigned flags, T *&cur, T *&po, int j1,
                    int j0, bool sample_src) {
    cudaEvent_t ev = prof_mark(ctx);
    T *c0 = cur, *p0 = po;
    auto body = [&]() -> esi_status {
        T *c = c0, *q = p0;
        for (int j = j1; j > j0; --j) {
            a.cur = c;
            a.po = q;
            a.n = j - 1;
            a.tin = j - 1;
            a.nout = j - 1;
            a.tout = (sample_src && j <= ctx->nt - 1) ? j : -1;
            a.slot_r = (j - 1) - j0;
            esi_status e = step<T>(ctx, flags, a, j < j1);
            if (e != ESI_OK) return e;
            std::swap(c, q);
        }
        return ESI_OK;
    };
    esi_status e;
    if (ctx->use_graphs && j1 - j0 >= GRAPH_MIN_STEPS) {
        auto key = loop_key(a, flags, -1, j0, j1, sample_src, c0, p0);
        if (!graph_replay(ctx, key, e)) e = graph_capture(ctx, std::move(key), body);
    } else {
        e = body();
    }
    if (e != ESI_OK) return e;
    if ((j1 - j0) & 1) std::swap(cur, po);
    prof_close(ctx, ev, step_name(ctx, flags), step_bpc(ctx, flags, a.nf), j1 - j0,
               (long long)(j1 - j0) * ctx->prof_active * ctx->N);
    return ESI_OK;
}

template <typename T>
esi_status adjoint_impl(esi_ctx *ctx, const void *traces, void *ext_out, void *wav_out,
                        bool pitched_out = false, const int *active = nullptr) {
    ctx->prof_active = ctx->ns;
    esi_status e = ensure_states<T>(ctx, true);
    if (e != ESI_OK) return e;
    CK(cudaMemsetAsync(ctx->a0.p, 0, ctx->a0.n, ctx->st));
    CK(cudaMemsetAsync(ctx->a1.p, 0, ctx->a1.n, ctx->st));
    StepArgs<T> a = base_args<T>(ctx);
    a.active = active;
    unsigned flags = F_PT;
    a.inj = inj_view<T>(ctx->inj_rec);
    a.inj_trace = reinterpret_cast<const T *>(traces);
    if (ext_out) {
        flags |= F_OUT;
        a.fout = reinterpret_cast<T *>(ext_out);
        // caller fields are dense; the CG right-hand side goes to an internal pitched vector
        a.opx = pitched_out ? ctx->px : ctx->g.nx;
        a.oplane = pitched_out ? ctx->sst : ctx->N;
        a.ofst = a.oplane * ctx->nt;
    }
    if (wav_out) {
        flags |= F_SMP;
        a.smp = smp_view<T>(ctx->smp_src);
        a.smp_out = reinterpret_cast<T *>(wav_out);
    }
    T *cur = ctx->a0.as<T>(), *po = ctx->a1.as<T>();
    e = adj_loop<T>(ctx, a, flags, cur, po, ctx->nt, 0, wav_out != nullptr);
    if (e != ESI_OK) return e;
    if (wav_out)
        CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, a.smp_out, 0, ctx->st));
    return ESI_OK;
}

// ------------------------------------------------------------------ gradient
// A compressed checkpoint holds u_n and the difference u_n - u_{n-1}, each in the two-level
// code of vec.cu (even cells plus the residual against their interpolation, FP16 or BF16
// with per-shot scales).  Between two steps at several samples per period the difference
// is a small fraction of u (about omega dt), so rounding u_{n-1} on its own would leave the
// recomputed leapfrog a velocity error far above the format's precision; rebuilding
// u_{n-1} = u_n - (u_n - u_{n-1}) from the decoded u_n keeps the difference accurate
// relative to itself.  Layout of ctx->ckpt for nseg segments: the fine parts
// [nseg][2][ns][sst], then the coarse parts [nseg][2][ns][csst] (uint16 codes); of
// ctx->ckpt_scale: the fine scales [nseg][2][ns], then the coarse ones.
template <typename T>
esi_status ckpt_store(esi_ctx *ctx, int kind, int nseg, int slot, const T *cur, const T *prev) {
    const long long len = ctx->sst;
    const int ns = ctx->ns;
    const T *src[2] = {cur, prev};
    const long long clen = ckpt_coarse_size(ctx->g.nz, ctx->g.ny, ctx->g.nx);
    const long long nsh = (long long)nseg * 2 * ns;   // shot states per part
    for (int h = 0; h < 2; ++h) {
        const long long idx = (long long)(2 * slot + h) * ns;  // in units of shot states
        if (kind == ESI_CKPT_F32) {
            CK(cudaMemcpyAsync(ctx->ckpt.as<T>() + idx * len, src[h], ns * len * sizeof(T),
                               cudaMemcpyDeviceToDevice, ctx->st));
        } else {
            uint16_t *codes = ctx->ckpt.as<uint16_t>();
            float *sc = ctx->ckpt_scale.as<float>();
            CKL(launch_ckpt_encode<T>(cur, h ? prev : nullptr, ns, ctx->g.nz, ctx->g.ny,
                                      ctx->g.nx, ctx->px, len, kind, ctx->absbits.as<unsigned>(),
                                      codes + idx * len, codes + nsh * len + idx * clen, sc + idx,
                                      sc + nsh + idx, ctx->st));
        }
    }
    return ESI_OK;
}

template <typename T>
esi_status ckpt_load(esi_ctx *ctx, int kind, int nseg, int slot, T *cur, T *prev) {
    const long long len = ctx->sst;
    const int ns = ctx->ns;
    T *dst[2] = {cur, prev};
    const long long clen = ckpt_coarse_size(ctx->g.nz, ctx->g.ny, ctx->g.nx);
    const long long nsh = (long long)nseg * 2 * ns;
    for (int h = 0; h < 2; ++h) {
        const long long idx = (long long)(2 * slot + h) * ns;
        if (kind == ESI_CKPT_F32) {
            CK(cudaMemcpyAsync(dst[h], ctx->ckpt.as<T>() + idx * len, ns * len * sizeof(T),
                               cudaMemcpyDeviceToDevice, ctx->st));
        } else {
            // u_n first; then u_{n-1} = (decoded u_n) - (decoded difference)
            const uint16_t *codes = ctx->ckpt.as<uint16_t>();
            const float *sc = ctx->ckpt_scale.as<float>();
            CKL(launch_ckpt_decode<T>(codes + idx * len, codes + nsh * len + idx * clen, sc + idx,
                                      sc + nsh + idx, ns, ctx->g.nz, ctx->g.ny, ctx->g.nx, ctx->px,
                                      len, kind, h ? cur : nullptr, dst[h], ctx->st));
        }
    }
    return ESI_OK;
}

template <typename T>
esi_status gradient_impl(esi_ctx *ctx, const void *wavelet, const void *ext, const void *dobs,
                         const void *adj, const esi_grad_opts *o, void *grad, double *misfit) {
    const long long N = ctx->N;
    const int ns = ctx->ns, nt = ctx->nt;
    ctx->prof_active = ns;
    esi_status e = ensure_states<T>(ctx, true);
    if (e != ESI_OK) return e;
    CK(ctx->gacc.ensure((size_t)ns * ctx->sst * sizeof(T)));
    CK(cudaMemsetAsync(ctx->gacc.p, 0, (size_t)ns * ctx->sst * sizeof(T), ctx->st));
    const T eps = T(o->eps > 0 ? o->eps : ctx->g.dx);
    double extra = 1.0;
    if (o->mode == ESI_GRAD_SADDLE_POINT || o->mode == ESI_GRAD_WRI_SADDLE) {
        if (!ext) return ctx->fail(ESI_ERR_ARG, "saddle-point gradient needs the extended source q");
        const bool wri = o->mode == ESI_GRAD_WRI_SADDLE;
        if (wri && !wavelet) return ctx->fail(ESI_ERR_ARG, "the WRI gradient needs the point sources f");
        CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        a.ext = reinterpret_cast<const T *>(ext);
        a.grad = ctx->gacc.as<T>();
        a.eps = eps;
        unsigned flags = F_EXT | F_SAD;
        if (wri) {   // u = A^{-1}(f + q), adjoint field beta q (B = I)
            flags |= F_PT;
            a.unit_b = 1;
            a.inj = inj_view<T>(ctx->inj_src);
            a.inj_trace = reinterpret_cast<const T *>(wavelet);
        }
        // with the observed data, the objective at (m, q) from the same run: Eq. "esi"
        // (WRI: "wrimisfit"), 1/2 ||R u - d||^2 + beta/2 ||B q||^2 (B = 1 for WRI)
        const bool want_J = misfit && dobs;
        if (want_J) {
            CK(ctx->traces.ensure(std::max<size_t>((size_t)ctx->total_rec * nt * sizeof(T), 16)));
            flags |= F_SMP;
            a.smp = smp_view<T>(ctx->smp_rec);
            a.smp_out = ctx->traces.as<T>();
        }
        T *cur = ctx->u0.as<T>(), *po = ctx->u1.as<T>();
        e = fwd_loop<T>(ctx, a, flags, cur, po, 0, nt);
        if (e != ESI_OK) return e;
        extra = -o->beta;
        if (want_J) {
            T *tr = ctx->traces.as<T>();
            CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, tr, nt - 1, ctx->st));
            const int nblk = 1024;
            CK(ctx->part.ensure(sizeof(double) * (size_t)nblk * std::max(ns, 1)));
            CK(ctx->scal.ensure(sizeof(double) * (1 + ns)));
            double *sc = ctx->scal.as<double>();
            CKL(launch_residual<T>(tr, reinterpret_cast<const T *>(dobs),
                                   (long long)ctx->total_rec * nt, ctx->part.as<double>(), nblk,
                                   ctx->st));
            CKL(launch_reduce_partials(ctx->part.as<double>(), nblk, 1, sc, ctx->st));
            CK(ctx->pb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
            CKL(launch_b2_maps<T>(ctx->pb2.as<T>(), nullptr, ns, ctx->g.nz, ctx->g.ny, ctx->g.nx,
                                  ctx->px, T(o->beta), eps, T(ctx->g.dx),
                                  ctx->src_pos.as<double>(), wri ? 1 : 0, ctx->st));
            CKL(launch_penalty<T>(reinterpret_cast<const T *>(ext), ctx->pb2.as<T>(), ns, nt,
                                  (long long)ctx->g.nz * ctx->g.ny, ctx->g.nx, ctx->px, ctx->sst,
                                  ctx->part.as<double>(), nblk, ctx->st));
            CKL(launch_reduce_partials(ctx->part.as<double>(), nblk, ns, sc + 1, ctx->st));
            std::vector<double> h(1 + ns);
            CK(cudaMemcpyAsync(h.data(), sc, sizeof(double) * (1 + ns), cudaMemcpyDeviceToHost,
                               ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
            double J = h[0];
            for (int s = 0; s < ns; ++s) J += h[1 + s];
            *misfit = J;
        }
    } else {
        if (!wavelet && !ext) return ctx->fail(ESI_ERR_ARG, "no source given");
        if (!adj && !dobs) return ctx->fail(ESI_ERR_ARG, "need observed data or an adjoint source");
        const int K = std::max(1, o->ckpt_every);
        const int nseg = (nt + K - 1) / K;
        const int kind = o->ckpt_kind;
        if (kind == ESI_CKPT_F32) {
            CK(ctx->ckpt.ensure((size_t)nseg * 2 * ns * ctx->sst * sizeof(T)));
        } else {   // fine + coarse 16-bit codes, two scales per shot state
            const long long clen = ckpt_coarse_size(ctx->g.nz, ctx->g.ny, ctx->g.nx);
            CK(ctx->ckpt.ensure((size_t)nseg * 2 * ns * (ctx->sst + clen) * 2));
        }
        CK(ctx->ckpt_scale.ensure(sizeof(float) * nseg * 2 * ns * 2));
        CK(ctx->absbits.ensure(sizeof(unsigned) * ns * 2));
        CK(ctx->stash.ensure((size_t)K * ns * ctx->sst * sizeof(T)));
        CK(ctx->traces.ensure(std::max<size_t>((size_t)ctx->total_rec * nt * sizeof(T), 16)));
        // 1) forward with checkpoints (u_{n0}, u_{n0-1}) at n0 = k K, traces into scratch
        CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        unsigned fflags = 0;
        if (wavelet) {
            fflags |= F_PT;
            a.inj = inj_view<T>(ctx->inj_src);
            a.inj_trace = reinterpret_cast<const T *>(wavelet);
        }
        if (ext) {
            fflags |= F_EXT;
            a.ext = reinterpret_cast<const T *>(ext);
        }
        T *tr = ctx->traces.as<T>();
        T *cur = ctx->u0.as<T>(), *po = ctx->u1.as<T>();
        a.smp = smp_view<T>(ctx->smp_rec);  // in VJP mode the traces are not used
        a.smp_out = tr;
        for (int sg = 0; sg < nseg; ++sg) {
            const int n0 = sg * K, n1 = std::min(nt, n0 + K);
            e = ckpt_store<T>(ctx, kind, nseg, sg, cur, po);
            if (e != ESI_OK) return e;
            if (adj && sg + 1 == nseg) break;  // the last segment is recomputed anyway
            e = fwd_loop<T>(ctx, a, fflags | F_SMP, cur, po, n0, n1);
            if (e != ESI_OK) return e;
        }
        const T *eres = reinterpret_cast<const T *>(adj);
        if (!adj) {
            CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, tr, nt - 1, ctx->st));
            const long long len = ctx->total_rec * nt;
            const int nblk = 1024;
            CK(ctx->part.ensure(sizeof(double) * nblk));
            CK(ctx->scal.ensure(sizeof(double) * 8));
            CKL(launch_residual<T>(tr, reinterpret_cast<const T *>(dobs), len, ctx->part.as<double>(),
                                   nblk, ctx->st));
            CKL(launch_reduce_partials(ctx->part.as<double>(), nblk, 1, ctx->scal.as<double>(), ctx->st));
            eres = tr;
        }
        // 2) backward: per segment, recompute with stash, then adjoint with correlation
        CK(cudaMemsetAsync(ctx->a0.p, 0, ctx->a0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->a1.p, 0, ctx->a1.n, ctx->st));
        T *acur = ctx->a0.as<T>(), *apo = ctx->a1.as<T>();
        StepArgs<T> b = base_args<T>(ctx);
        b.inj = inj_view<T>(ctx->inj_rec);
        b.inj_trace = eres;
        b.grad = ctx->gacc.as<T>();
        b.stash_r = ctx->stash.as<T>();
        a.stash_w = ctx->stash.as<T>();
        a.smp = SmpList<T>();
        for (int sg = nseg - 1; sg >= 0; --sg) {
            const int n0 = sg * K, n1 = std::min(nt, n0 + K);
            T *fc = ctx->u0.as<T>(), *fp = ctx->u1.as<T>();
            e = ckpt_load<T>(ctx, kind, nseg, sg, fc, fp);
            if (e != ESI_OK) return e;
            e = fwd_loop<T>(ctx, a, fflags | F_STW, fc, fp, n0, n1);
            if (e != ESI_OK) return e;
            e = adj_loop<T>(ctx, b, F_PT | F_GRD, acur, apo, n1, n0, false);
            if (e != ESI_OK) return e;
        }
        if (misfit && !adj) {
            CK(cudaMemcpyAsync(misfit, ctx->scal.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
        }
    }
    (void)N;
    CKL(launch_grad_finalize<T>(ctx->gacc.as<T>(), ns, ctx->sst, ctx->cc.as<T>(), ctx->g.nz,
                                ctx->g.ny, ctx->g.nx, ctx->px, ctx->dt, ctx->g.dx, extra, o->param,
                                reinterpret_cast<T *>(grad), ctx->st));
    if (misfit && !adj && o->mode == ESI_GRAD_ADJOINT_STATE) return check_dev_err(ctx);
    return ESI_OK;
}

// ------------------------------------------------------------------ DTFT
template <typename T>
esi_status dft_impl(esi_ctx *ctx, const void *wavelet, const void *ext, const double *freqs,
                    int nf, void *out, int kind, float *scales, void *traces) {
    if (nf <= 0 || !freqs || !out) return ctx->fail(ESI_ERR_ARG, "need frequencies and an output");
    if (kind != ESI_DFT_C64 && kind != ESI_DFT_C32_HALF)
        return ctx->fail(ESI_ERR_ARG, "unknown DTFT output kind");
    if (kind == ESI_DFT_C32_HALF && !scales)
        return ctx->fail(ESI_ERR_ARG, "half output needs a scales array");
    // accumulators in the internal pitched layout [ns][nf][sst][2]
    const size_t accb = (size_t)ctx->ns * nf * ctx->sst * 2 * sizeof(T);
    CK(ctx->dftacc.ensure(accb));
    T *acc = ctx->dftacc.as<T>();
    CK(cudaMemsetAsync(acc, 0, accb, ctx->st));
    esi_status e = forward_impl<T>(ctx, wavelet, ext, traces, freqs, nf, acc);
    if (e != ESI_OK) return e;
    const int half = kind == ESI_DFT_C32_HALF;
    CK(ctx->absbits.ensure(sizeof(unsigned) * ctx->ns * nf));
    CK(ctx->ckpt_scale.ensure(std::max(ctx->ckpt_scale.n, sizeof(float) * ctx->ns * nf)));
    CKL(launch_dft_output<T>(acc, ctx->sst, ctx->g.nz * ctx->g.ny, ctx->g.nx, ctx->px, ctx->ns, nf,
                             half, out, ctx->absbits.as<unsigned>(), ctx->ckpt_scale.as<float>(),
                             ctx->st));
    if (half) {
        CK(cudaMemcpyAsync(scales, ctx->ckpt_scale.p, sizeof(float) * ctx->ns * nf,
                           cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return ESI_OK;
}

// ------------------------------------------------------------------ CG (Algorithm 1)
// Per shot: x0 = 0, r0 = b = S^T d, p0 = z0; alpha = rho / <p, A p>; x += alpha p;
// r -= alpha A p; stop when ||r_{k+1}|| < tol ||r_0|| or k = max_iter - 1; beta = rho_new /
// rho; p = z + beta p, where z = r (no preconditioner, Algorithm 1 as printed) or
// z = r / (lambda B^2) (diagonal preconditioner) and rho = <r, z>.  The work vectors r, p,
// A p live in the internal pitched layout; x is the caller's dense q_out.
// WRI (the CG section: the same CG with B = I and its own right-hand side, Eq. "normalwri"): with
// wri_wavelet the annihilator is the identity and the right-hand side is S^T (d - S f), f the
// point sources; the rest of Algorithm 1 is unchanged.
template <typename T>
esi_status cg_impl(esi_ctx *ctx, double lambda, double tol, int max_iter, const void *dobs,
                   void *q_out, int precond, double eps_in, esi_cg_report *rep,
                   const void *wri_wavelet = nullptr) {
    const int unit_b = wri_wavelet != nullptr;
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    const int ns = ctx->ns, nt = ctx->nt;
    const long long plen = ctx->sst * nt;                       // pitched vector per shot
    const long long rows = (long long)nt * ctx->g.nz * ctx->g.ny;
    bool learned = precond == ESI_PC_LEARNED;
    if (precond != ESI_PC_NONE && precond != ESI_PC_DIAG && !learned)
        return ctx->fail(ESI_ERR_ARG, "unknown preconditioner");
    if (learned && unit_b)
        return ctx->fail(ESI_ERR_UNSUPPORTED, "the learned preconditioner serves the ESI system");
    if (learned && (!ctx->pc || sizeof(T) != 4 || ctx->g.ndim != 2))
        return ctx->fail(ESI_ERR_UNSUPPORTED,
                         "the learned preconditioner needs esi_pc_load on a 2D FP32 context");
    if (precond != ESI_PC_NONE && !(lambda > 0))
        return ctx->fail(ESI_ERR_ARG, "preconditioning needs lambda > 0");
    if (max_iter < 1) return ctx->fail(ESI_ERR_ARG, "max_iter must be >= 1");
    esi_status e = ensure_states<T>(ctx, true);
    if (e != ESI_OK) return e;
    const size_t vb = (size_t)ns * plen * sizeof(T);
    CK(ctx->cg_r.ensure(vb));
    CK(ctx->cg_p.ensure(vb));
    CK(ctx->cg_ap.ensure(vb));
    CK(ctx->traces.ensure(std::max<size_t>((size_t)ctx->total_rec * nt * sizeof(T), 16)));
    // <p, A p> partials of the adjoint half: one per warp of a 2D tile, one per 3D block
    const int nblk_step = ctx->g.ndim == 2 ? ctx->ntx * ctx->ntz * (NT2 / 32)
                                            : ctx->ntx * ctx->nty * ctx->nzc;
    const int nblk_vec = 1216;  // 8 x 152 SMs
    const size_t npart = (size_t)ns * std::max(nblk_step, nblk_vec);
    CK(ctx->part.ensure(sizeof(double) * npart));
    CK(ctx->part2.ensure(sizeof(double) * npart));
    // device scalars: rho[ns] rr[ns] rho_new[ns] pap[ns] alpha[ns] beta[ns] | active[ns] bad[ns]
    CK(ctx->scal.ensure(sizeof(double) * 6 * ns + sizeof(int) * 2 * ns));
    double *rho = ctx->scal.as<double>(), *rr = rho + ns, *rho_new = rr + ns, *pap = rho_new + ns,
           *alpha = pap + ns, *beta = alpha + ns;
    int *active = reinterpret_cast<int *>(beta + ns), *bad = active + ns;
    T *x = reinterpret_cast<T *>(q_out), *r = ctx->cg_r.as<T>(), *p = ctx->cg_p.as<T>(),
      *ap = ctx->cg_ap.as<T>(), *tr = ctx->traces.as<T>();
    const T eps = T(eps_in > 0 ? eps_in : ctx->g.dx);
    const T pc = precond != ESI_PC_NONE ? T(lambda) : T(0);
    double *rz_part = pc > T(0) ? ctx->part2.as<double>() : nullptr;
    // lambda B^2 (and its inverse for the diagonal preconditioner), once per solve
    CK(ctx->pb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
    T *ipb2 = nullptr;
    if (pc > T(0)) {
        CK(ctx->ipb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
        ipb2 = ctx->ipb2.as<T>();
    }
    CKL(launch_b2_maps<T>(ctx->pb2.as<T>(), ipb2, ns, ctx->g.nz, ctx->g.ny, ctx->g.nx, ctx->px,
                          T(lambda), eps, T(ctx->g.dx), ctx->src_pos.as<double>(), unit_b, ctx->st));
    const int nzny = ctx->g.nz * ctx->g.ny;
    // learned preconditioner, per shot: z = s + theta up2(U(pack(s))), s = r / (lambda B^2),
    // with the flexible (Polak-Ribiere) beta = -alpha <z_{k+1}, A p_k> / <z_k, r_k>.  theta = 1
    // while the network keeps <z, r> >= <s, r> / 2 (> 0) on every active shot; the first time
    // it does not on any shot, the solve drops the network (theta = 0) and every shot restarts
    // its directions from the diagonal preconditioner (beta = 0) for the rest of the solve.
    // (Dropping it per shot, or damping theta, measured more iterations: the shots that keep
    // the network longer restart later.)
    const int ng = (nt + 15) / 16, hc = (ctx->g.nz + 1) / 2, wc = (ctx->g.nx + 1) / 2;
    const long long nimg = (long long)ns * ng, img_elems = (long long)hc * wc * 16;
    // pc_dev: the four partial-dot arrays [4][ns][nblk_vec], their per-shot sums [4][ns]
    // (<s, r>, <y, r>, <s, A p>, <y, A p>) and theta [ns]
    std::vector<int> h_active(ns, 1), h_bad(ns, 0), iters(ns, 0);
    std::vector<char> h_conv(ns, 0);
    double *pc_part = nullptr, *pc_dots = nullptr, *pc_theta = nullptr;
    std::vector<double> h_rho(ns), h_rhon(ns), h_za(ns), h_alpha(ns), h_beta(ns, 0.0);
    std::vector<double> h_dots(4 * (size_t)ns), h_theta(ns, 1.0);
    std::vector<char> h_restart(ns, 0);
    if (learned) {
        CK(ctx->pc_img.ensure((size_t)nimg * img_elems * 2));
        CK(ctx->pc_y.ensure((size_t)nimg * img_elems * 4));
        CK(ctx->pc_dev.ensure(sizeof(double) * (4 * (size_t)ns * nblk_vec + 4 * (size_t)ns + ns)));
        pc_part = ctx->pc_dev.as<double>();
        pc_dots = pc_part + 4 * (size_t)ns * nblk_vec;
        pc_theta = pc_dots + 4 * (size_t)ns;
    }
    // theta, <z, r> and <z, A p_prev> per active shot from the four sums on the host
    auto pc_combine = [&](bool with_ap) {
        bool fail = false;
        for (int s = 0; s < ns; ++s) {
            if (!h_active[s]) continue;
            const double sr = h_dots[s], yr = h_dots[ns + s], ya = h_dots[3 * ns + s];
            fail |= !std::isfinite(yr) || (with_ap && !std::isfinite(ya)) || sr + yr < 0.5 * sr;
        }
        if (fail) ctx->pc_fallbacks++;
        for (int s = 0; s < ns; ++s) {
            if (!h_active[s]) continue;
            const double sr = h_dots[s], yr = h_dots[ns + s], sa = h_dots[2 * ns + s],
                         ya = h_dots[3 * ns + s];
            h_restart[s] = fail;
            h_theta[s] = fail ? 0.0 : 1.0;
            h_rhon[s] = fail ? sr : sr + yr;
            h_za[s] = with_ap ? sa + h_theta[s] * ya : 0.0;
        }
    };
    const long long pc_cells = (long long)ns * nt * ctx->N;   // fine space-time elements
    auto apply_learned = [&](const T *ap_prev) -> esi_status {
        const float *rf = reinterpret_cast<const float *>(r);
        cudaEvent_t pev = prof_mark(ctx);
        CKL(pcnet::pack_launch(rf, reinterpret_cast<const float *>(ipb2), ctx->pc_img.as<__nv_bfloat16>(),
                               ns, nt, ctx->g.nz, ctx->g.nx, ctx->px, ctx->sst, 1, 0, ctx->st));
        // reads r, writes the 2 x 2-averaged BF16 image (1/8 of a float per element)
        prof_close(ctx, pev, "pc_pack", 4.5, 1, pc_cells);
        pev = prof_mark(ctx);
        for (long long i0 = 0; i0 < nimg; i0 += ctx->pc_batch) {
            const int nb = (int)std::min<long long>(ctx->pc_batch, nimg - i0);
            CK(pcnet_forward(ctx->pc, ctx->pc_img.as<__nv_bfloat16>() + i0 * img_elems, nb,
                             ctx->pc_y.as<float>() + i0 * img_elems, ctx->st, true));
            ctx->launches += 13;
        }
        // the network's own input and output streams (0.5 + 1 byte per element); its
        // intermediate activations are not counted
        prof_close(ctx, pev, "pc_net", 1.5, (nimg + ctx->pc_batch - 1) / ctx->pc_batch * 13, pc_cells);
        pev = prof_mark(ctx);
        CKL(pcnet::pc_dots_launch(rf, reinterpret_cast<const float *>(ap_prev),
                                  reinterpret_cast<const float *>(ipb2), ctx->pc_y.as<float>(),
                                  pc_part, nblk_vec, ns, nt, ctx->g.nz, ctx->g.nx, ctx->px,
                                  ctx->sst, active, ctx->st));
        CKL(launch_reduce_partials(pc_part, nblk_vec, 4 * ns, pc_dots, ctx->st));
        CK(cudaMemcpyAsync(h_dots.data(), pc_dots, sizeof(double) * 4 * ns, cudaMemcpyDeviceToHost,
                           ctx->st));
        // reads r, A p and the coarse correction (a quarter of a float per element)
        prof_close(ctx, pev, "pc_dots", ap_prev ? 9.0 : 5.0, ap_prev ? 3 : 2, pc_cells);
        return ESI_OK;
    };
    CK(cudaMemsetAsync(bad, 0, sizeof(int) * ns, ctx->st));
    CK(cudaMemsetAsync(alpha, 0, sizeof(double) * ns, ctx->st));
    CK(cudaMemsetAsync(x, 0, (size_t)ns * ctx->N * nt * sizeof(T), ctx->st));
    if (unit_b) {
        // WRI: the data residual d - S f of the point sources replaces d
        const long long tl = (long long)ctx->total_rec * nt;
        CK(ctx->wri_res.ensure(std::max<size_t>((size_t)tl * sizeof(T), 16)));
        e = forward_impl<T>(ctx, wri_wavelet, nullptr, ctx->wri_res.p, nullptr, 0, nullptr);
        if (e != ESI_OK) return e;
        CKL(launch_sub_from<T>(ctx->wri_res.as<T>(), reinterpret_cast<const T *>(dobs), tl, ctx->st));
        dobs = ctx->wri_res.p;
    }
    // b = S^T d, written straight into r (x0 = 0, r0 = b)
    e = adjoint_impl<T>(ctx, dobs, r, nullptr, true);
    if (e != ESI_OK) return e;
    // ||r0||^2 and rho0 = <r0, z0>: the update pass with alpha = 0 (p = Ap = r)
    CKL(launch_cg_update<T>(x, r, r, r, rows, ctx->g.nx, ctx->px, ns, alpha, nullptr,
                            ctx->part.as<double>(), rz_part, nblk_vec, ipb2, ctx->sst, nzny,
                            ctx->st));
    CKL(launch_reduce_partials(ctx->part.as<double>(), nblk_vec, ns, rr, ctx->st));
    CKL(launch_reduce_partials(rz_part ? rz_part : ctx->part.as<double>(), nblk_vec, ns, rho, ctx->st));
    CK(cudaMemsetAsync(active, 0xff, sizeof(int) * ns, ctx->st));  // nonzero: all shots
    if (learned) {   // z_0, theta_0 and rho_0 = <z_0, r_0>
        e = apply_learned(nullptr);
        if (e != ESI_OK) return e;
        CK(cudaStreamSynchronize(ctx->st));
        pc_combine(false);
        h_rho = h_rhon;
        CK(cudaMemcpyAsync(rho, h_rho.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(pc_theta, h_theta.data(), sizeof(double) * ns, cudaMemcpyHostToDevice,
                           ctx->st));
    }
    std::vector<double> rr0(ns), rrn(ns);
    CK(cudaMemcpyAsync(rr0.data(), rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    const int hist_cap = rep ? rep->max_hist : 0;
    for (int s = 0; s < ns; ++s)
        if (!(rr0[s] > 0)) h_active[s] = 0;  // b = 0: x = 0 is exact
    CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
    double ms_mv = 0, ms_vec = 0, ms_pc = 0;
    // phase split of each iteration, timed on the device: [ev0, ev1) the product, [ev1, ev3)
    // the vector work, of which [ev2, ev3) the learned preconditioner
    struct Events {
        cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
        ~Events() {
            for (auto x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    for (auto &x : ev.e) CK(cudaEventCreate(&x));
    int k;
    bool any_bad = false;
    for (k = 0; k < max_iter; ++k) {
        CK(cudaEventRecord(ev.e[0], ctx->st));
        ctx->prof_active = 0;
        for (int s = 0; s < ns; ++s) ctx->prof_active += h_active[s];
        // forward half of the product, fused with p = z + beta p (p0 = z0)
        CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        a.active = active;
        a.cg_r = r;
        a.cg_p = p;
        a.cg_beta = beta;
        a.cg_first = k == 0;
        a.cg_pc = pc;
        a.ipb2 = ipb2;
        a.eps = eps;
        if (learned) {
            a.pc_y = ctx->pc_y.as<float>();
            a.pc_theta = pc_theta;
            a.pc_ng = ng;
            a.pc_hc = hc;
            a.pc_wc = wc;
            a.cg_beta = beta;
        }
        a.smp = smp_view<T>(ctx->smp_rec);
        a.smp_out = tr;
        T *cur = ctx->u0.as<T>(), *po = ctx->u1.as<T>();
        e = fwd_loop<T>(ctx, a, F_CGP | F_SMP, cur, po, 0, nt);
        if (e != ESI_OK) return e;
        CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, tr, nt - 1, ctx->st));
        // adjoint half: Ap = S^T (S p) + lambda B^2 p, with <p, Ap> partials
        CK(cudaMemsetAsync(ctx->a0.p, 0, ctx->a0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->a1.p, 0, ctx->a1.n, ctx->st));
        CK(cudaMemsetAsync(ctx->part.p, 0, sizeof(double) * (size_t)ns * nblk_step, ctx->st));
        StepArgs<T> b = base_args<T>(ctx);
        b.active = active;
        b.inj = inj_view<T>(ctx->inj_rec);
        b.inj_trace = tr;
        b.ap = ap;
        b.ap_p = p;
        b.dot_part = ctx->part.as<double>();
        b.pen = T(lambda);
        b.pb2 = ctx->pb2.as<T>();
        b.eps = eps;
        T *acur = ctx->a0.as<T>(), *apo = ctx->a1.as<T>();
        e = adj_loop<T>(ctx, b, F_PT | F_AP, acur, apo, nt, 0, false);
        if (e != ESI_OK) return e;
        CKL(launch_reduce_partials(ctx->part.as<double>(), nblk_step, ns, pap, ctx->st));
        CKL(launch_cg_alpha(rho, pap, alpha, bad, active, ns, ctx->st));
        CK(cudaEventRecord(ev.e[1], ctx->st));
        cudaEvent_t pev = prof_mark(ctx);
        CKL(launch_cg_update<T>(x, r, p, ap, rows, ctx->g.nx, ctx->px, ns, alpha, active,
                                ctx->part.as<double>(), learned ? nullptr : rz_part, nblk_vec,
                                learned ? nullptr : ipb2, ctx->sst, nzny, ctx->st));
        prof_close(ctx, pev, "cg_update", (6.0 + 0.0) * sizeof(T), 1,
                   (long long)ctx->prof_active * ctx->N * nt);
        CKL(launch_reduce_partials(ctx->part.as<double>(), nblk_vec, ns, rr, ctx->st));
        if (learned) {
            CK(cudaEventRecord(ev.e[2], ctx->st));
            e = apply_learned(ap);
            if (e != ESI_OK) return e;
            CK(cudaMemcpyAsync(h_alpha.data(), alpha, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
            CK(cudaEventRecord(ev.e[3], ctx->st));
        } else {
            CKL(launch_reduce_partials(rz_part ? rz_part : ctx->part.as<double>(), nblk_vec, ns,
                                       rho_new, ctx->st));
        }
        if (!learned) CK(cudaEventRecord(ev.e[3], ctx->st));
        CK(cudaMemcpyAsync(rrn.data(), rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(h_bad.data(), bad, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if ((e = check_dev_err(ctx)) != ESI_OK) return e;
        {
            float m01 = 0, m13 = 0, m23 = 0;
            CK(cudaEventElapsedTime(&m01, ev.e[0], ev.e[1]));
            CK(cudaEventElapsedTime(&m13, ev.e[1], ev.e[3]));
            if (learned) CK(cudaEventElapsedTime(&m23, ev.e[2], ev.e[3]));
            ms_mv += m01;
            ms_vec += m13 - m23;
            ms_pc += m23;
        }
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            if (!h_active[s]) continue;
            if (h_bad[s]) {
                any_bad = true;
                h_active[s] = 0;
                continue;
            }
            iters[s] = k + 1;
            const double rel = std::sqrt(rrn[s] / rr0[s]);
            if (rep && rep->rel_res && k < hist_cap) rep->rel_res[(size_t)s * hist_cap + k] = rel;
            const bool met = std::sqrt(rrn[s]) < tol * std::sqrt(rr0[s]);
            h_conv[s] = met;
            if (met || k == max_iter - 1)
                h_active[s] = 0;  // exit loop for this shot (Algorithm 1's stopping test)
            else
                any = true;
        }
        if (!any) break;
        CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
        if (learned) {
            pc_combine(true);
            for (int s = 0; s < ns; ++s) {
                h_beta[s] = h_active[s] && !h_restart[s] ? -h_alpha[s] * h_za[s] / h_rho[s] : 0.0;
                if (h_active[s]) h_rho[s] = h_rhon[s];
            }
            CK(cudaMemcpyAsync(beta, h_beta.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(rho, h_rho.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(pc_theta, h_theta.data(), sizeof(double) * ns, cudaMemcpyHostToDevice,
                               ctx->st));
            // once every active shot has dropped the network the solve is the diagonal PCG
            // (rho already holds <s, r>): stop running the network
            bool any_net = false;
            for (int s = 0; s < ns; ++s) any_net |= h_active[s] && h_theta[s] > 0.0;
            if (!any_net) learned = false;
        } else {
            CKL(launch_cg_beta(rho, rho_new, beta, active, ns, ctx->st));
        }
    }
    // judged on each shot's own last residual (the device partials of frozen shots are reused)
    bool conv = true;
    for (int s = 0; s < ns; ++s)
        if (rr0[s] > 0 && !(iters[s] > 0 && h_conv[s])) conv = false;
    if (rep) {
        int mx = 0;
        for (int s = 0; s < ns; ++s) {
            mx = std::max(mx, iters[s]);
            if (rep->iters) rep->iters[s] = iters[s];
        }
        rep->iters_max = mx;
        rep->converged = conv ? 1 : 0;
        rep->ms_matvec = ms_mv;
        rep->ms_vector = ms_vec;
        rep->ms_precond = ms_pc;
        rep->ms_total = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    }
    if (any_bad) return ctx->fail(ESI_ERR_BREAKDOWN, "CG breakdown: p^T A p <= 0 or non-finite");
    return conv ? ESI_OK : ESI_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ data-space CG
// The section "Switching from the wavefield to data space": Algorithm 1 on Eq. "wd",
//   (I + K) w = K d,   K = S (lambda B^2)^{-1} S^T,
// for the synthetic data w (traces layout), then Eq. "q": q = (lambda B^2)^{-1} S^T (d - w).
// K e is one adjoint modelling of e (its space-time field kept in a pitched context buffer)
// and one forward modelling with that field times 1/(lambda B^2) as the extended source
// (the CG forward-half kernel with p = z = r / (lambda B^2), sampling at the receivers).
// The CG vectors are data vectors: per iteration no pass over space-time vectors remains
// besides the product's own field.  The nonzero spectrum of I + K is that of the diagonally
// preconditioned wavefield system, so the iteration counts match the diagonal PCG.
template <typename T>
esi_status dscg_impl(esi_ctx *ctx, double lambda, double tol, int max_iter, const void *dobs,
                     void *q_out, void *w_out, double eps_in, esi_cg_report *rep) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    const int ns = ctx->ns, nt = ctx->nt;
    if (!(lambda > 0)) return ctx->fail(ESI_ERR_ARG, "the data-space form needs lambda > 0");
    if (max_iter < 1) return ctx->fail(ESI_ERR_ARG, "max_iter must be >= 1");
    esi_status e = ensure_states<T>(ctx, true);
    if (e != ESI_OK) return e;
    const long long plen = ctx->sst * nt;
    const long long dl = (long long)ctx->total_rec * nt;      // data vector length
    CK(ctx->cg_r.ensure((size_t)ns * plen * sizeof(T)));       // the adjoint field S^T e
    CK(ctx->cg_p.ensure((size_t)ns * plen * sizeof(T)));       // the scaled source (written)
    CK(ctx->dsv.ensure((size_t)5 * std::max<long long>(dl, 4) * sizeof(T)));
    T *F = ctx->cg_r.as<T>(), *Fs = ctx->cg_p.as<T>();
    T *x = ctx->dsv.as<T>(), *r = x + dl, *p = r + dl, *kp = p + dl, *db = kp + dl;
    const T eps = T(eps_in > 0 ? eps_in : ctx->g.dx);
    CK(ctx->pb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
    CK(ctx->ipb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
    T *ipb2 = ctx->ipb2.as<T>();
    CKL(launch_b2_maps<T>(ctx->pb2.as<T>(), ipb2, ns, ctx->g.nz, ctx->g.ny, ctx->g.nx, ctx->px,
                          T(lambda), eps, T(ctx->g.dx), ctx->src_pos.as<double>(), 0, ctx->st));
    // shot segments of the data vectors
    std::vector<long long> seg(ns + 1);
    for (int s = 0; s <= ns; ++s) seg[s] = ctx->rec_off[s] * (long long)nt;
    CK(upload(ctx->dseg, seg, ctx->st));
    const long long *dseg = ctx->dseg.as<long long>();
    const int nb = DVEC_NBLK;
    CK(ctx->part.ensure(sizeof(double) * (size_t)ns * nb));
    // device scalars: rr[ns] pap[ns] alpha[ns] beta[ns] rrn[ns] | active[ns] bad[ns]
    CK(ctx->scal.ensure(sizeof(double) * 5 * ns + sizeof(int) * 2 * ns));
    double *rr = ctx->scal.as<double>(), *pap = rr + ns, *alpha = pap + ns, *beta = alpha + ns,
           *rrn = beta + ns;
    int *active = reinterpret_cast<int *>(rrn + ns), *bad = active + ns;
    CK(cudaMemsetAsync(active, 0xff, sizeof(int) * ns, ctx->st));
    CK(cudaMemsetAsync(bad, 0, sizeof(int) * ns, ctx->st));
    // out = K e for the active shots
    auto apply_K = [&](const T *ein, T *out) -> esi_status {
        esi_status st = adjoint_impl<T>(ctx, ein, F, nullptr, true, active);
        if (st != ESI_OK) return st;
        CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        a.active = active;
        a.cg_r = F;
        a.cg_p = Fs;
        a.cg_beta = beta;
        a.cg_first = 1;           // p = z = F / (lambda B^2)
        a.cg_pc = T(lambda);
        a.ipb2 = ipb2;
        a.eps = eps;
        a.smp = smp_view<T>(ctx->smp_rec);
        a.smp_out = out;
        T *cur = ctx->u0.as<T>(), *po = ctx->u1.as<T>();
        st = fwd_loop<T>(ctx, a, F_CGP | F_SMP, cur, po, 0, nt);
        if (st != ESI_OK) return st;
        CKL(launch_sample_global<T>(a.smp, cur, ctx->sst, out, nt - 1, ctx->st));
        return ESI_OK;
    };
    // right-hand side K d; x0 = 0, r0 = p0 = K d
    e = apply_K(reinterpret_cast<const T *>(dobs), db);
    if (e != ESI_OK) return e;
    CK(cudaMemsetAsync(x, 0, dl * sizeof(T), ctx->st));
    CK(cudaMemcpyAsync(r, db, dl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(p, db, dl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemsetAsync(alpha, 0, sizeof(double) * ns, ctx->st));
    CKL(launch_dvec_update<T>(x, r, p, p, dseg, alpha, nullptr, ctx->part.as<double>(), ns, ctx->st));
    CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rr, ctx->st));
    std::vector<double> rr0(ns), h_rrn(ns);
    std::vector<int> h_active(ns, 1), h_bad(ns, 0), iters(ns, 0);
    std::vector<char> h_conv(ns, 0);
    CK(cudaMemcpyAsync(rr0.data(), rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int s = 0; s < ns; ++s)
        if (!(rr0[s] > 0)) h_active[s] = 0;
    CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
    const int hist_cap = rep ? rep->max_hist : 0;
    double ms_mv = 0, ms_vec = 0;
    struct Events {
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        ~Events() {
            for (auto z : e)
                if (z) cudaEventDestroy(z);
        }
    } ev;
    for (auto &z : ev.e) CK(cudaEventCreate(&z));
    bool any_bad = false;
    for (int k = 0; k < max_iter; ++k) {
        ctx->prof_active = 0;
        for (int s = 0; s < ns; ++s) ctx->prof_active += h_active[s];
        CK(cudaEventRecord(ev.e[0], ctx->st));
        e = apply_K(p, kp);                                      // kp = K p
        if (e != ESI_OK) return e;
        CK(cudaEventRecord(ev.e[1], ctx->st));
        CKL(launch_dvec_ident_dot<T>(kp, p, dseg, active, ctx->part.as<double>(), ns, ctx->st));
        CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, pap, ctx->st));
        CKL(launch_cg_alpha(rr, pap, alpha, bad, active, ns, ctx->st));
        CKL(launch_dvec_update<T>(x, r, p, kp, dseg, alpha, active, ctx->part.as<double>(), ns, ctx->st));
        CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rrn, ctx->st));
        CK(cudaEventRecord(ev.e[2], ctx->st));
        CK(cudaMemcpyAsync(h_rrn.data(), rrn, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(h_bad.data(), bad, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if ((e = check_dev_err(ctx)) != ESI_OK) return e;
        float m01 = 0, m12 = 0;
        CK(cudaEventElapsedTime(&m01, ev.e[0], ev.e[1]));
        CK(cudaEventElapsedTime(&m12, ev.e[1], ev.e[2]));
        ms_mv += m01;
        ms_vec += m12;
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            if (!h_active[s]) continue;
            if (h_bad[s]) {
                any_bad = true;
                h_active[s] = 0;
                continue;
            }
            iters[s] = k + 1;
            if (rep && rep->rel_res && k < hist_cap)
                rep->rel_res[(size_t)s * hist_cap + k] = std::sqrt(h_rrn[s] / rr0[s]);
            const bool met = std::sqrt(h_rrn[s]) < tol * std::sqrt(rr0[s]);
            h_conv[s] = met;
            if (met || k == max_iter - 1)
                h_active[s] = 0;   // Algorithm 1's stopping test, per shot
            else
                any = true;
        }
        if (!any) break;
        CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
        CKL(launch_cg_beta(rr, rrn, beta, active, ns, ctx->st));
        CKL(launch_dvec_xpby<T>(p, r, dseg, beta, active, ns, ctx->st));
    }
    // q = (lambda B^2)^{-1} S^T (d - w), every shot
    CK(cudaMemsetAsync(active, 0xff, sizeof(int) * ns, ctx->st));
    CK(cudaMemcpyAsync(r, x, dl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CKL(launch_sub_from<T>(r, reinterpret_cast<const T *>(dobs), dl, ctx->st));
    e = adjoint_impl<T>(ctx, r, F, nullptr, true);
    if (e != ESI_OK) return e;
    CKL(launch_scale_to_dense<T>(reinterpret_cast<T *>(q_out), F, ipb2, ns, nt,
                                 ctx->g.nz * ctx->g.ny, ctx->g.nx, ctx->px, ctx->sst, ctx->st));
    if (w_out)
        CK(cudaMemcpyAsync(w_out, x, dl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    bool conv = true;
    int mx = 0;
    for (int s = 0; s < ns; ++s) {
        if (rr0[s] > 0 && !(iters[s] > 0 && h_conv[s])) conv = false;
        mx = std::max(mx, iters[s]);
    }
    if (rep) {
        for (int s = 0; s < ns && rep->iters; ++s) rep->iters[s] = iters[s];
        rep->iters_max = mx;
        rep->converged = conv ? 1 : 0;
        rep->ms_matvec = ms_mv;
        rep->ms_vector = ms_vec;
        rep->ms_precond = 0;
        rep->ms_total = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    }
    if (any_bad) return ctx->fail(ESI_ERR_BREAKDOWN, "CG breakdown: p^T (I + K) p <= 0 or non-finite");
    return conv ? ESI_OK : ESI_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ frequency-domain ESI
// The section "Frequency domain inversion by time domain modelling": CG on Eq. "normaldtft",
//   F (S^T S + lambda B^T B) F^H qbar / nt = F S^T d,
// over nf complex frequency slices per shot (qbar pitched [ns][nf][sst][2]; the CG works in
// the real representation, where the Hermitian positive definite operator is symmetric
// positive definite).  One product: for the real and the imaginary part of the time series
// F^H qbar / nt, a forward modelling whose source is synthesised block by block from qbar
// (Eq. "idtft"), then an adjoint modelling of its traces whose output is folded block by
// block into the frequency slices (Eq. "dtft"; the imaginary part's twiddles turned by j);
// then lambda B^2 G qbar per cell (G = F F^H / nt).  No space-time vector is stored: the
// sources and the adjoint output pass through dft_k-step stashes.
template <typename T>
esi_status fdcg_impl(esi_ctx *ctx, double lambda, double tol, int max_iter, const void *dobs,
                     const double *freqs, int nf, int precond, void *qbar_out, double eps_in,
                     esi_cg_report *rep) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    const int ns = ctx->ns, nt = ctx->nt, K = ctx->dft_k;
    if (nf < 1 || nf > FD_MAXF)
        return ctx->fail(ESI_ERR_ARG, "need 1 .. " + std::to_string(FD_MAXF) + " frequencies");
    for (int m = 0; m < nf; ++m)
        if (!std::isfinite(freqs[m])) return ctx->fail(ESI_ERR_ARG, "frequencies must be finite");
    if (!(lambda > 0)) return ctx->fail(ESI_ERR_ARG, "the frequency-domain form needs lambda > 0");
    if (max_iter < 1) return ctx->fail(ESI_ERR_ARG, "max_iter must be >= 1");
    if (precond != ESI_PC_NONE && precond != ESI_PC_DIAG)
        return ctx->fail(ESI_ERR_UNSUPPORTED, "the frequency-domain CG takes no or the diagonal preconditioner");
    const bool pc = precond == ESI_PC_DIAG;
    esi_status e = ensure_states<T>(ctx, true);
    if (e != ESI_OK) return e;
    const long long vl = (long long)ns * nf * ctx->sst * 2;   // one complex unknown vector
    CK(ctx->fdv.ensure((size_t)6 * vl * sizeof(T)));
    T *X = ctx->fdv.as<T>(), *R = X + vl, *P = R + vl, *AP = P + vl, *Bv = AP + vl, *Z = Bv + vl;
    // source stash [ns][K][sst] and the scratch the fused kernel writes its source to
    CK(ctx->fdsrc.ensure((size_t)2 * ns * K * ctx->sst * sizeof(T)));
    T *src = ctx->fdsrc.as<T>(), *psc = src + (size_t)ns * K * ctx->sst;
    CK(ctx->dftsnap.ensure((size_t)K * ns * ctx->sst * sizeof(T)));
    const long long tl = std::max<long long>((long long)ctx->total_rec * nt, 4);
    CK(ctx->fdtr.ensure((size_t)tl * sizeof(T)));
    T *tr = ctx->fdtr.as<T>();
    const T eps = T(eps_in > 0 ? eps_in : ctx->g.dx);
    CK(ctx->pb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
    T *ipb2 = nullptr;   // 1 / (lambda B^2) for the diagonal preconditioner
    if (pc) {
        CK(ctx->ipb2.ensure((size_t)ns * ctx->sst * sizeof(T)));
        ipb2 = ctx->ipb2.as<T>();
    }
    CKL(launch_b2_maps<T>(ctx->pb2.as<T>(), ipb2, ns, ctx->g.nz, ctx->g.ny, ctx->g.nx, ctx->px,
                          T(lambda), eps, T(ctx->g.dx), ctx->src_pos.as<double>(), 0, ctx->st));
    // twiddle tables [part][n][m][2]: synthesis of the real part (cos, sin) / nt and of the
    // imaginary part (-sin, cos) / nt; folding of a real series (cos, sin) and of an
    // imaginary one (-sin, cos); the Gram matrix G[m][k] = 1/nt sum_n e^{j (ph_m - ph_k) n}
    std::vector<T> syn((size_t)2 * nt * nf * 2), fold((size_t)2 * nt * nf * 2);
    std::vector<double> G((size_t)nf * nf * 2, 0.0);
    for (int n = 0; n < nt; ++n)
        for (int m = 0; m < nf; ++m) {
            const double ph = 2.0 * M_PI * freqs[m] * n * ctx->dt, c = std::cos(ph), sn = std::sin(ph);
            const size_t o = ((size_t)n * nf + m) * 2, o1 = (size_t)nt * nf * 2 + o;
            syn[o] = T(c / nt), syn[o + 1] = T(sn / nt);
            syn[o1] = T(-sn / nt), syn[o1 + 1] = T(c / nt);
            fold[o] = T(c), fold[o + 1] = T(sn);
            fold[o1] = T(-sn), fold[o1 + 1] = T(c);
            for (int k = 0; k < nf; ++k) {
                const double d = 2.0 * M_PI * (freqs[m] - freqs[k]) * n * ctx->dt;
                G[(m * nf + k) * 2] += std::cos(d) / nt;
                G[(m * nf + k) * 2 + 1] += std::sin(d) / nt;
            }
        }
    CK(upload(ctx->fdsyn, syn, ctx->st));
    CK(upload(ctx->fdfold, fold, ctx->st));
    CK(upload(ctx->fdG, G, ctx->st));
    const T *syn_d = ctx->fdsyn.as<T>(), *fold_d = ctx->fdfold.as<T>();
    const double *G_d = ctx->fdG.as<double>();
    std::vector<long long> seg(ns + 1);   // shot segments of the real-representation vectors
    for (int s = 0; s <= ns; ++s) seg[s] = (long long)s * nf * ctx->sst * 2;
    CK(upload(ctx->dseg, seg, ctx->st));
    const long long *dseg = ctx->dseg.as<long long>();
    const int nb = DVEC_NBLK;
    CK(ctx->part.ensure(sizeof(double) * (size_t)ns * nb));
    CK(ctx->scal.ensure(sizeof(double) * 7 * ns + sizeof(int) * 2 * ns));
    double *rr = ctx->scal.as<double>(), *pap = rr + ns, *alpha = pap + ns, *beta = alpha + ns,
           *rrn = beta + ns, *rz = rrn + ns, *rzn = rz + ns;   // rz: Re <r, z> (preconditioned)
    int *active = reinterpret_cast<int *>(rzn + ns), *bad = active + ns;
    CK(cudaMemsetAsync(active, 0xff, sizeof(int) * ns, ctx->st));
    CK(cudaMemsetAsync(bad, 0, sizeof(int) * ns, ctx->st));
    const double es = double(sizeof(T));
    const unsigned aflags = ctx->g.ndim == 2 ? (F_PT | F_SMP | F_DFT) : (F_PT | F_DFT);
    // out += F S^T traces, the j-th part's twiddles (part 1: the series times j)
    auto adjoint_fold = [&](const T *traces, int part, T *out) -> esi_status {
        cudaEvent_t ev = prof_mark(ctx);
        CK(cudaMemsetAsync(ctx->a0.p, 0, ctx->a0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->a1.p, 0, ctx->a1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        a.active = active;
        a.inj = inj_view<T>(ctx->inj_rec);
        a.inj_trace = traces;
        a.smp = smp_view<T>(ctx->smp_rec);   // no sampling: tout < 0
        a.stash_w = ctx->dftsnap.as<T>();
        a.nf = nf;
        a.twid = fold_d + (size_t)part * nt * nf * 2;
        a.dft = out;
        T *c0 = ctx->a0.as<T>(), *p0 = ctx->a1.as<T>();
        auto body = [&]() -> esi_status {
            T *c = c0, *q = p0;
            for (int jhi = nt; jhi > 0;) {
                const int jlo = std::max(0, jhi - K);
                for (int j = jhi; j > jlo; --j) {
                    a.cur = c;
                    a.po = q;
                    a.n = j - 1;
                    a.tin = j - 1;
                    a.nout = j - 1;
                    a.tout = -1;
                    a.slot_w = (j - 1) - jlo;   // slots in time order within the block
                    esi_status st = step<T>(ctx, aflags, a, j < nt);
                    if (st != ESI_OK) return st;
                    std::swap(c, q);
                }
                CKL(launch_dft_block<T>(a.stash_w, jhi - jlo, ns, ctx->sst, ctx->g.nx, ctx->px, nf,
                                        a.twid + (size_t)jlo * nf * 2, out, ctx->st));
                jhi = jlo;
            }
            return ESI_OK;
        };
        esi_status st;
        if (ctx->use_graphs && nt >= GRAPH_MIN_STEPS) {
            auto key = loop_key(a, aflags, -3, part, nt, false, c0, p0);
            if (!graph_replay(ctx, key, st)) st = graph_capture(ctx, std::move(key), body);
        } else {
            st = body();
        }
        if (st != ESI_OK) return st;
        prof_close(ctx, ev, step_name(ctx, aflags) + "+dft_block",
                   step_bpc(ctx, aflags, nf) + es + 4.0 * nf * es / K, nt + (nt + K - 1) / K,
                   (long long)nt * ctx->prof_active * ctx->N);
        return ESI_OK;
    };
    // traces of the forward modelling whose source is part `part` of F^H qb / nt
    auto forward_synth = [&](const T *qb, int part) -> esi_status {
        cudaEvent_t ev = prof_mark(ctx);
        CK(cudaMemsetAsync(ctx->u0.p, 0, ctx->u0.n, ctx->st));
        CK(cudaMemsetAsync(ctx->u1.p, 0, ctx->u1.n, ctx->st));
        StepArgs<T> a = base_args<T>(ctx);
        a.active = active;
        a.cg_r = src;
        a.cg_p = psc;
        a.cg_first = 1;   // the source is the stash slot itself
        a.fstp = (long long)K * ctx->sst;
        a.smp = smp_view<T>(ctx->smp_rec);
        a.smp_out = tr;
        a.ext = qb;       // not read by the step; part of the loop key
        a.nf = nf;
        a.twid = syn_d + (size_t)part * nt * nf * 2;
        T *c0 = ctx->u0.as<T>(), *p0 = ctx->u1.as<T>();
        auto body = [&]() -> esi_status {
            T *c = c0, *q = p0;
            for (int n0 = 0; n0 < nt; n0 += K) {
                const int n1 = std::min(nt, n0 + K);
                CKL(launch_idft_block<T>(qb, n1 - n0, K, ns, ctx->sst, nf,
                                         a.twid + (size_t)n0 * nf * 2, src, ctx->st));
                for (int n = n0; n < n1; ++n) {
                    a.cur = c;
                    a.po = q;
                    a.n = n - n0;   // the stash slot
                    a.tin = n;
                    a.tout = n - 1;
                    esi_status st = step<T>(ctx, F_CGP | F_SMP, a, n > 0);
                    if (st != ESI_OK) return st;
                    std::swap(c, q);
                }
            }
            CKL(launch_sample_global<T>(a.smp, c, ctx->sst, tr, nt - 1, ctx->st));
            return ESI_OK;
        };
        esi_status st;
        if (ctx->use_graphs && nt >= GRAPH_MIN_STEPS) {
            auto key = loop_key(a, F_CGP | F_SMP, +3, part, nt, false, c0, p0);
            if (!graph_replay(ctx, key, st)) st = graph_capture(ctx, std::move(key), body);
        } else {
            st = body();
        }
        if (st != ESI_OK) return st;
        prof_close(ctx, ev, step_name(ctx, F_CGP | F_SMP) + "+idft_block",
                   step_bpc(ctx, F_CGP | F_SMP, 0) + es + 2.0 * nf * es / K, nt + (nt + K - 1) / K,
                   (long long)nt * ctx->prof_active * ctx->N);
        return ESI_OK;
    };
    // out = F (S^T S + lambda B^2) F^H qb / nt, with the partials of Re <qb, out>
    auto apply_M = [&](const T *qb, T *out) -> esi_status {
        CK(cudaMemsetAsync(out, 0, vl * sizeof(T), ctx->st));
        for (int part = 0; part < 2; ++part) {
            esi_status st = forward_synth(qb, part);
            if (st != ESI_OK) return st;
            st = adjoint_fold(tr, part, out);
            if (st != ESI_OK) return st;
        }
        CKL(launch_fd_b2g_dot<T>(out, qb, ctx->pb2.as<T>(), G_d, nf, ns, ctx->sst, active,
                                 ctx->part.as<double>(), ctx->st));
        return ESI_OK;
    };
    ctx->prof_active = ns;
    // right-hand side F S^T d
    CK(cudaMemsetAsync(Bv, 0, vl * sizeof(T), ctx->st));
    e = adjoint_fold(reinterpret_cast<const T *>(dobs), 0, Bv);
    if (e != ESI_OK) return e;
    CK(cudaMemsetAsync(X, 0, vl * sizeof(T), ctx->st));
    CK(cudaMemcpyAsync(R, Bv, vl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(P, Bv, vl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemsetAsync(alpha, 0, sizeof(double) * ns, ctx->st));
    CKL(launch_dvec_update<T>(X, R, P, P, dseg, alpha, nullptr, ctx->part.as<double>(), ns, ctx->st));
    CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rr, ctx->st));
    if (pc) {   // z0 = M^{-1} r0, p0 = z0
        CKL(launch_fd_precond<T>(Z, R, ipb2, nf, ns, ctx->sst, nullptr, ctx->part.as<double>(), ctx->st));
        CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rz, ctx->st));
        CK(cudaMemcpyAsync(P, Z, vl * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    }
    std::vector<double> rr0(ns), h_rrn(ns);
    std::vector<int> h_active(ns, 1), h_bad(ns, 0), iters(ns, 0);
    std::vector<char> h_conv(ns, 0);
    CK(cudaMemcpyAsync(rr0.data(), rr, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    for (int s = 0; s < ns; ++s)
        if (!(rr0[s] > 0)) h_active[s] = 0;   // b = 0: qbar = 0 is exact
    CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
    const int hist_cap = rep ? rep->max_hist : 0;
    double ms_mv = 0, ms_vec = 0;
    struct Events {
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        ~Events() {
            for (auto z : e)
                if (z) cudaEventDestroy(z);
        }
    } ev;
    for (auto &z : ev.e) CK(cudaEventCreate(&z));
    bool any_bad = false;
    for (int k = 0; k < max_iter; ++k) {
        ctx->prof_active = 0;
        for (int s = 0; s < ns; ++s) ctx->prof_active += h_active[s];
        if (ctx->prof_active == 0) break;
        CK(cudaEventRecord(ev.e[0], ctx->st));
        e = apply_M(P, AP);
        if (e != ESI_OK) return e;
        CK(cudaEventRecord(ev.e[1], ctx->st));
        CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, pap, ctx->st));
        CKL(launch_cg_alpha(pc ? rz : rr, pap, alpha, bad, active, ns, ctx->st));
        CKL(launch_dvec_update<T>(X, R, P, AP, dseg, alpha, active, ctx->part.as<double>(), ns, ctx->st));
        CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rrn, ctx->st));
        CK(cudaEventRecord(ev.e[2], ctx->st));
        CK(cudaMemcpyAsync(h_rrn.data(), rrn, sizeof(double) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaMemcpyAsync(h_bad.data(), bad, sizeof(int) * ns, cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        if ((e = check_dev_err(ctx)) != ESI_OK) return e;
        float m01 = 0, m12 = 0;
        CK(cudaEventElapsedTime(&m01, ev.e[0], ev.e[1]));
        CK(cudaEventElapsedTime(&m12, ev.e[1], ev.e[2]));
        ms_mv += m01;
        ms_vec += m12;
        bool any = false;
        for (int s = 0; s < ns; ++s) {
            if (!h_active[s]) continue;
            if (h_bad[s]) {
                any_bad = true;
                h_active[s] = 0;
                continue;
            }
            iters[s] = k + 1;
            if (rep && rep->rel_res && k < hist_cap)
                rep->rel_res[(size_t)s * hist_cap + k] = std::sqrt(h_rrn[s] / rr0[s]);
            const bool met = std::sqrt(h_rrn[s]) < tol * std::sqrt(rr0[s]);
            h_conv[s] = met;
            if (met || k == max_iter - 1)
                h_active[s] = 0;
            else
                any = true;
        }
        if (!any) break;
        CK(cudaMemcpyAsync(active, h_active.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, ctx->st));
        if (pc) {   // z = M^{-1} r, beta = <r', z'> / <r, z>, p = z + beta p
            CKL(launch_fd_precond<T>(Z, R, ipb2, nf, ns, ctx->sst, active, ctx->part.as<double>(),
                                     ctx->st));
            CKL(launch_reduce_partials(ctx->part.as<double>(), nb, ns, rzn, ctx->st));
            CKL(launch_cg_beta(rz, rzn, beta, active, ns, ctx->st));
            CKL(launch_dvec_xpby<T>(P, Z, dseg, beta, active, ns, ctx->st));
        } else {
            CKL(launch_cg_beta(rr, rrn, beta, active, ns, ctx->st));
            CKL(launch_dvec_xpby<T>(P, R, dseg, beta, active, ns, ctx->st));
        }
    }
    // qbar out: pitched complex slices -> dense [ns][nf][N][2]
    CKL(launch_dft_output<T>(X, ctx->sst, ctx->g.nz * ctx->g.ny, ctx->g.nx, ctx->px, ns, nf, 0,
                             qbar_out, nullptr, nullptr, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    bool conv = true;
    int mx = 0;
    for (int s = 0; s < ns; ++s) {
        if (rr0[s] > 0 && !(iters[s] > 0 && h_conv[s])) conv = false;
        mx = std::max(mx, iters[s]);
    }
    if (rep) {
        for (int s = 0; s < ns && rep->iters; ++s) rep->iters[s] = iters[s];
        rep->iters_max = mx;
        rep->converged = conv ? 1 : 0;
        rep->ms_matvec = ms_mv;
        rep->ms_vector = ms_vec;
        rep->ms_precond = 0;
        rep->ms_total = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    }
    if (any_bad) return ctx->fail(ESI_ERR_BREAKDOWN, "CG breakdown: Re <p, M p> <= 0 or non-finite");
    return conv ? ESI_OK : ESI_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ outer loop
// Algorithm "nestedloop": inner CG solve, objective and saddle-point gradient in v, L-BFGS
// direction, projected Armijo backtracking, penalty schedule.  Model vectors are dense [N]
// in the field precision; their dot products and maxima are reduced in double on the host
// (block partials summed in a fixed order).
template <typename T>
esi_status invert_impl(esi_ctx *ctx, const esi_invert_opts *o, const void *wavelet,
                       const void *dobs, void *vel, void *gwork, esi_invert_report *rep) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    const bool wri = o->mode == ESI_GRAD_WRI_SADDLE;
    if (o->mode != ESI_GRAD_SADDLE_POINT && !wri)
        return ctx->fail(ESI_ERR_ARG, "mode must be the ESI or the WRI saddle-point mode");
    if (wri && !wavelet) return ctx->fail(ESI_ERR_ARG, "WRI needs the point sources f");
    if (o->n_outer < 0 || o->n_cg < 1 || o->memory < 1 || o->memory > 64 || o->max_ls < 1 ||
        !(o->beta0 > 0) || !(o->growth > 0) || !(o->c1 > 0 && o->c1 < 1) || !(o->step_frac > 0) ||
        !(o->vmin > 0) || !(o->vmax > o->vmin) || !std::isfinite(o->vmax) || !(o->cg_tol >= 0))
        return ctx->fail(ESI_ERR_ARG, "bad outer-loop options");
    if (rep && rep->max_iters < o->n_outer)
        return ctx->fail(ESI_ERR_ARG, "report arrays shorter than n_outer");
    if (!wri && o->precond == ESI_PC_LEARNED && !ctx->pc)
        return ctx->fail(ESI_ERR_ARG, "the learned preconditioner is not loaded");
    const long long N = ctx->N;
    const int M = o->memory;
    CK(ctx->invq.ensure((size_t)ctx->ns * ctx->nt * N * sizeof(T)));
    CK(ctx->invv.ensure((size_t)(6 + 2 * M) * N * sizeof(T)));
    T *q = ctx->invq.as<T>(), *V = ctx->invv.as<T>();
    T *x = reinterpret_cast<T *>(vel), *gw = reinterpret_cast<T *>(gwork);
    T *g = V, *gt = V + N, *xt = V + 2 * N, *d = V + 3 * N, *sv = V + 4 * N, *yv = V + 5 * N;
    T *Sp = V + 6 * N, *Yp = V + (6 + M) * N;   // pair slots
    const int nblk = 256;
    CK(ctx->invpart.ensure(sizeof(double) * nblk));
    std::vector<double> hp(nblk);
    auto reduce_host = [&](bool is_max, double &out) -> esi_status {
        CK(cudaMemcpyAsync(hp.data(), ctx->invpart.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost,
                           ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        out = 0;
        for (double v : hp) out = is_max ? std::max(out, v) : out + v;
        return ESI_OK;
    };
    auto dot = [&](const T *a, const T *b, double &out) -> esi_status {
        CKL(launch_mdot<T>(a, b, N, ctx->invpart.as<double>(), nblk, ctx->st));
        return reduce_host(false, out);
    };
    auto amax = [&](const T *a, double &out) -> esi_status {
        CKL(launch_mamax<T>(a, N, ctx->invpart.as<double>(), nblk, ctx->st));
        return reduce_host(true, out);
    };
    auto lin = [&](T *z, double al, const T *xx, double be, const T *yy, bool clamp) -> esi_status {
        CKL(launch_mlincomb<T>(z, al, xx, be, yy, N, clamp ? o->vmin : 0.0, clamp ? o->vmax : 0.0,
                               ctx->st));
        return ESI_OK;
    };
    int evals = 0, cg_total = 0;
    esi_grad_opts go{};
    go.mode = o->mode;
    go.param = ESI_PARAM_V;
    go.ckpt_every = 1;
    go.ckpt_kind = ESI_CKPT_F32;
    go.eps = o->eps;
    // J and g (into g_out) at the model m, through the entry points: with shot groups
    // (esi_set_shot_groups) the inner solve and the gradient run on them
    auto eval = [&](const T *m, double beta, T *g_out, double &J) -> esi_status {
        esi_status st = esi_set_velocity(ctx, m);
        if (st != ESI_OK) return st;
        std::vector<int> its(ctx->ns);
        esi_cg_report cr{};
        cr.iters = its.data();
        st = wri ? esi_wri_solve(ctx, beta, o->cg_tol, o->n_cg, wavelet, dobs, q, &cr)
                 : esi_cg_solve(ctx, beta, o->cg_tol, o->n_cg, dobs, q, o->precond, o->eps, &cr);
        if (st != ESI_OK && st != ESI_ERR_NOT_CONVERGED) return st;
        cg_total += cr.iters_max;
        go.beta = beta;
        st = esi_gradient(ctx, wri ? wavelet : nullptr, q, dobs, nullptr, &go, gw, &J);
        if (st != ESI_OK) return st;
        if (o->reduce) {
            CK(cudaStreamSynchronize(ctx->st));
            if (o->reduce(o->reduce_user, &J, gw, N) != 0)
                return ctx->fail(ESI_ERR_ARG, "the reduce callback failed");
        }
        CK(cudaMemcpyAsync(g_out, gw, N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
        ++evals;
        return ESI_OK;
    };
    auto beta_of = [&](int i) { return o->beta0 * std::pow(o->growth, i); };
    std::vector<double> rho, gam;   // per stored pair (oldest first): 1 / y^T s, s^T y / y^T y
    std::vector<int> slot;          // pair -> slot index
    int next_slot = 0;
    double J = 0, Jt = 0;
    esi_status e = eval(x, beta_of(0), g, J);
    if (e != ESI_OK) return e;
    int stop = 0, done = 0;
    for (int i = 0; i < o->n_outer; ++i) {
        const double beta = beta_of(i);
        if (i > 0 && beta != beta_of(i - 1)) {
            if ((e = eval(x, beta, g, J)) != ESI_OK) return e;
            rho.clear(), gam.clear(), slot.clear();
        }
        if (rep && rep->beta) rep->beta[i] = beta;
        if (rep && rep->J_start) rep->J_start[i] = J;
        // two-loop recursion: d = -H g
        if ((e = lin(d, 1.0, g, 0.0, nullptr, false)) != ESI_OK) return e;
        const int np = int(slot.size());
        std::vector<double> a(np);
        for (int k = np - 1; k >= 0; --k) {
            double sd;
            if ((e = dot(Sp + (size_t)slot[k] * N, d, sd)) != ESI_OK) return e;
            a[k] = rho[k] * sd;
            if ((e = lin(d, 1.0, d, -a[k], Yp + (size_t)slot[k] * N, false)) != ESI_OK) return e;
        }
        if (np > 0 && (e = lin(d, gam[np - 1], d, 0.0, nullptr, false)) != ESI_OK) return e;
        for (int k = 0; k < np; ++k) {
            double yd;
            if ((e = dot(Yp + (size_t)slot[k] * N, d, yd)) != ESI_OK) return e;
            const double b = rho[k] * yd;
            if ((e = lin(d, 1.0, d, a[k] - b, Sp + (size_t)slot[k] * N, false)) != ESI_OK) return e;
        }
        if ((e = lin(d, -1.0, d, 0.0, nullptr, false)) != ESI_OK) return e;
        double gd;
        if ((e = dot(g, d, gd)) != ESI_OK) return e;
        bool have_pairs = np > 0;
        if (!(gd < 0)) {   // not a descent direction: steepest descent, memory cleared
            rho.clear(), gam.clear(), slot.clear();
            have_pairs = false;
            if ((e = lin(d, -1.0, g, 0.0, nullptr, false)) != ESI_OK) return e;
        }
        double alpha = 1.0;
        if (!have_pairs) {
            double dmax, xmax;
            if ((e = amax(d, dmax)) != ESI_OK) return e;
            if ((e = amax(x, xmax)) != ESI_OK) return e;
            if (!(dmax > 0)) {
                stop = 2;
                break;
            }
            alpha = o->step_frac * xmax / dmax;
        }
        bool ok = false;
        int t = 0;
        for (t = 0; t < o->max_ls; ++t) {
            if ((e = lin(xt, 1.0, x, alpha, d, true)) != ESI_OK) return e;
            if ((e = eval(xt, beta, gt, Jt)) != ESI_OK) return e;
            if ((e = lin(sv, 1.0, xt, -1.0, x, false)) != ESI_OK) return e;
            double gs;
            if ((e = dot(g, sv, gs)) != ESI_OK) return e;
            if (Jt <= J + o->c1 * gs) {
                ok = true;
                break;
            }
            alpha *= 0.5;
        }
        if (rep && rep->trials) rep->trials[i] = std::min(t + 1, o->max_ls);
        if (!ok) {
            stop = 1;
            break;
        }
        // pair (s, y) = (xt - x, gt - g), kept on positive curvature
        if ((e = lin(yv, 1.0, gt, -1.0, g, false)) != ESI_OK) return e;
        double sy, yy, ss;
        if ((e = dot(sv, yv, sy)) != ESI_OK) return e;
        if ((e = dot(yv, yv, yy)) != ESI_OK) return e;
        if ((e = dot(sv, sv, ss)) != ESI_OK) return e;
        if (sy > 1e-12 * std::sqrt(ss) * std::sqrt(yy)) {
            int sl;
            if (int(slot.size()) == M) {   // drop the oldest, reuse its slot
                sl = slot.front();
                slot.erase(slot.begin());
                rho.erase(rho.begin());
                gam.erase(gam.begin());
            } else {
                sl = next_slot++;
            }
            CK(cudaMemcpyAsync(Sp + (size_t)sl * N, sv, N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
            CK(cudaMemcpyAsync(Yp + (size_t)sl * N, yv, N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
            slot.push_back(sl);
            rho.push_back(1.0 / sy);
            gam.push_back(sy / yy);
        }
        CK(cudaMemcpyAsync(x, xt, N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
        std::swap(g, gt);
        J = Jt;
        ++done;
        if (rep && rep->J_end) rep->J_end[i] = J;
        if (rep && rep->alpha) rep->alpha[i] = alpha;
    }
    // leave the context (and its shot groups) at the output model and the caller's gradient
    // at its gradient
    if ((e = esi_set_velocity(ctx, x)) != ESI_OK) return e;
    CK(cudaMemcpyAsync(gw, g, N * sizeof(T), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    if (rep) {
        rep->iters_done = done;
        rep->evaluations = evals;
        rep->cg_iters_total = cg_total;
        rep->stop_reason = stop;
        rep->ms_total = std::chrono::duration<double, std::milli>(clk::now() - t_start).count();
    }
    return check_dev_err(ctx);
}

template <typename T>
esi_status create_impl(esi_ctx *ctx, const void *vel) {
    CK(ctx->dev_err.ensure(sizeof(int)));
    CK(cudaMemsetAsync(ctx->dev_err.p, 0, sizeof(int), ctx->st));
    esi_status e = setup_model<T>(ctx, vel, true);
    if (e != ESI_OK) return e;
    e = setup_geometry<T>(ctx);
    if (e != ESI_OK) return e;
    CK(cudaStreamSynchronize(ctx->st));
    return ESI_OK;
}

}  // namespace

#define DISPATCH(ctx, call)                                          \
    ((ctx)->g.dtype == ESI_F64 ? call<double> : call<float>)

namespace {
// Runs fn(g, child) for every shot group, the first in the calling thread and the others in
// threads of their own, so that the groups' launches, host syncs and tails overlap.  Each
// group's stream first waits for the work queued so far on the context stream (the caller's
// inputs), and the context stream then waits for every group.  A failing group's status and
// message become the call's (ESI_ERR_NOT_CONVERGED only when no group failed otherwise).
template <typename Fn>
esi_status run_groups(esi_ctx *ctx, Fn &&fn) {
    const int G = (int)ctx->grp.size();
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaEventRecord(ctx->grp_ev[0], ctx->st));
    for (int g = 0; g < G; ++g) CK(cudaStreamWaitEvent(ctx->grp_st[g], ctx->grp_ev[0], 0));
    std::vector<esi_status> st(G, ESI_OK);
    std::vector<std::string> msg(G);
    auto one = [&](int g) {
        try {
            st[g] = fn(g, ctx->grp[g]);
        } catch (const std::exception &ex) {
            st[g] = ESI_ERR_CUDA;
            msg[g] = ex.what();
        }
    };
    std::vector<std::thread> th;
    for (int g = 1; g < G; ++g)
        th.emplace_back([&, g]() {
            if (cudaSetDevice(dev) != cudaSuccess) {
                st[g] = ESI_ERR_CUDA;
                msg[g] = "cudaSetDevice failed in a shot-group thread";
                return;
            }
            one(g);
        });
    one(0);
    for (auto &t : th) t.join();
    for (int g = 0; g < G; ++g) {
        CK(cudaEventRecord(ctx->grp_ev[1 + g], ctx->grp_st[g]));
        CK(cudaStreamWaitEvent(ctx->st, ctx->grp_ev[1 + g], 0));
    }
    esi_status out = ESI_OK;
    for (int g = 0; g < G; ++g) {
        if (st[g] == ESI_OK) continue;
        if (st[g] == ESI_ERR_NOT_CONVERGED) {
            out = ESI_ERR_NOT_CONVERGED;
            continue;
        }
        return ctx->fail(st[g], "shot group " + std::to_string(g) + ": " +
                                    (msg[g].empty() ? ctx->grp[g]->err : msg[g]));
    }
    return out;
}

// byte offset of shot s in a seismogram-layout buffer and in a [ns][nt][N] field
inline size_t trace_off(const esi_ctx *ctx, int s) {
    return (size_t)ctx->rec_off[s] * ctx->nt * ctx->esz;
}
inline size_t field_off(const esi_ctx *ctx, int s) {
    return (size_t)s * ctx->nt * ctx->N * ctx->esz;
}
template <typename P>
P *at(P *p, size_t bytes) {   // p + bytes, NULL stays NULL
    using B = typename std::conditional<std::is_const<P>::value, const char, char>::type;
    return p ? reinterpret_cast<P *>(reinterpret_cast<B *>(p) + bytes) : nullptr;
}

// A CG-type solve over the groups: solve(k, child, report of group k) with the caller's
// report arrays offset to the group's shots; the merged report has the per-shot entries of
// every group, the largest iteration count, convergence of all, the longest group's phase
// times and the wall clock of the whole call.
template <typename Solve>
esi_status run_group_solves(esi_ctx *ctx, esi_cg_report *report, Solve &&solve) {
    const auto t0 = std::chrono::steady_clock::now();
    const int G = (int)ctx->grp.size();
    std::vector<esi_cg_report> reps(G);
    const esi_status e = run_groups(ctx, [&](int k, esi_ctx *c) {
        const int s0 = ctx->grp_s0[k];
        esi_cg_report *r = nullptr;
        if (report) {
            reps[k] = *report;
            reps[k].iters = report->iters ? report->iters + s0 : nullptr;
            reps[k].rel_res = report->rel_res ? report->rel_res + (size_t)s0 * report->max_hist : nullptr;
            r = &reps[k];
        }
        return solve(k, c, r);
    });
    if (report && (e == ESI_OK || e == ESI_ERR_NOT_CONVERGED)) {
        report->iters_max = 0;
        report->converged = 1;
        report->ms_matvec = report->ms_vector = report->ms_precond = 0.0;
        for (const auto &r : reps) {
            report->iters_max = std::max(report->iters_max, r.iters_max);
            report->converged &= r.converged;
            report->ms_matvec = std::max(report->ms_matvec, r.ms_matvec);
            report->ms_vector = std::max(report->ms_vector, r.ms_vector);
            report->ms_precond = std::max(report->ms_precond, r.ms_precond);
        }
        report->ms_total =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return e;
}
}  // namespace

extern "C" {

ESI_API const char *esi_status_string(esi_status s) {
    switch (s) {
        case ESI_OK: return "ok";
        case ESI_ERR_ARG: return "invalid argument";
        case ESI_ERR_CFL: return "time step above the stability limit";
        case ESI_ERR_OOM: return "device allocation failed";
        case ESI_ERR_CUDA: return "CUDA error";
        case ESI_ERR_BREAKDOWN: return "CG breakdown";
        case ESI_ERR_TIMEOUT: return "device wait timed out";
        case ESI_ERR_NOT_CONVERGED: return "CG did not reach the tolerance";
        case ESI_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown status";
}

namespace {
thread_local std::string g_create_error;  // message of the last failed esi_create
}

ESI_API const char *esi_last_error(const esi_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

ESI_API long long esi_launch_count(const esi_ctx *ctx) {
    if (!ctx) return 0;
    long long n = ctx->launches;
    for (const auto *c : ctx->grp) n += c->launches;
    return n;
}

ESI_API esi_status esi_set_profiling(esi_ctx *ctx, int on) {
    if (!ctx) return ESI_ERR_ARG;
    cudaStreamSynchronize(ctx->st);
    for (auto &p : ctx->pending) {
        ctx->evpool.push_back(p.a);
        ctx->evpool.push_back(p.b);
    }
    ctx->pending.clear();
    ctx->stats.clear();
    ctx->prof = on != 0;
    for (auto *c : ctx->grp) esi_set_profiling(c, on);
    return ESI_OK;
}

ESI_API int esi_get_profile(esi_ctx *ctx, esi_kernel_stat *out, int max) {
    if (!ctx) return 0;
    cudaStreamSynchronize(ctx->st);
    for (auto &p : ctx->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        esi_ctx::Stat *st = nullptr;
        for (auto &x : ctx->stats)
            if (x.name == p.name) st = &x;
        if (!st) {
            ctx->stats.push_back(esi_ctx::Stat());
            st = &ctx->stats.back();
            st->name = p.name;
            st->bpc = p.bpc;
        }
        st->launches += p.launches;
        st->cells += p.cells;
        st->ms += ms;
        ctx->evpool.push_back(p.a);
        ctx->evpool.push_back(p.b);
    }
    ctx->pending.clear();
    // the shot groups' runs, merged by name (their times are per group stream: groups run
    // at the same time, so a merged time is the sum over groups of overlapping spans)
    for (auto *c : ctx->grp) {
        const int nc = esi_get_profile(c, nullptr, 0);
        std::vector<esi_kernel_stat> tmp(nc);
        esi_get_profile(c, tmp.data(), nc);
        for (const auto &k : tmp) {
            esi_ctx::Stat *st = nullptr;
            for (auto &x : ctx->stats)
                if (x.name == k.name) st = &x;
            if (!st) {
                ctx->stats.push_back(esi_ctx::Stat());
                st = &ctx->stats.back();
                st->name = k.name;
                st->bpc = k.bytes_per_cell;
            }
            st->launches += k.launches;
            st->cells += k.cells;
            st->ms += k.ms;
        }
        esi_set_profiling(c, c->prof);   // consumed: the group's stats start again
    }
    const int n = (int)ctx->stats.size();
    for (int i = 0; i < n && i < max && out; ++i) {
        std::memset(out[i].name, 0, sizeof(out[i].name));
        std::strncpy(out[i].name, ctx->stats[i].name.c_str(), sizeof(out[i].name) - 1);
        out[i].launches = ctx->stats[i].launches;
        out[i].cells = ctx->stats[i].cells;
        out[i].bytes_per_cell = ctx->stats[i].bpc;
        out[i].ms = ctx->stats[i].ms;
    }
    return n;
}

ESI_API esi_status esi_create(esi_ctx **out, const esi_grid *grid, const esi_geometry *geom,
                              const void *velocity_dev, double dt, int nt, void *stream) {
    g_create_error.clear();
    if (!out || !grid || !geom || !velocity_dev) return ESI_ERR_ARG;
    *out = nullptr;
    const esi_grid &g = *grid;
    if ((g.ndim != 2 && g.ndim != 3) || g.nz < 1 || g.nx < 1 || g.ny < 1 ||
        (g.ndim == 2 && g.ny != 1) || !(g.dx > 0) || g.nb < 0 ||
        (g.nb > 0 && !(g.sponge_R > 0 && g.sponge_R < 1)) ||
        (g.dtype != ESI_F32 && g.dtype != ESI_F64) || !(dt > 0) || nt < 1 || geom->ns < 1 ||
        !geom->src_xyz || !geom->rec_offset || (geom->rec_offset[geom->ns] > 0 && !geom->rec_xyz))
        return ESI_ERR_ARG;
    for (int s = 0; s < geom->ns; ++s)
        if (geom->rec_offset[s + 1] < geom->rec_offset[s]) return ESI_ERR_ARG;
    std::unique_ptr<esi_ctx> ctx(new esi_ctx());
    ctx->g = g;
    ctx->ns = geom->ns;
    ctx->nt = nt;
    ctx->dt = dt;
    ctx->st = reinterpret_cast<cudaStream_t>(stream);
    ctx->esz = g.dtype == ESI_F64 ? 8 : 4;
    ctx->N = (long long)g.nz * g.ny * g.nx;
    ctx->px = (g.nx + PITCH - 1) / PITCH * PITCH;
    ctx->sst = (long long)g.nz * g.ny * ctx->px;
    ctx->src_xyz.assign(geom->src_xyz, geom->src_xyz + 3 * geom->ns);
    ctx->rec_off.assign(geom->rec_offset, geom->rec_offset + geom->ns + 1);
    ctx->total_rec = ctx->rec_off[ctx->ns];
    ctx->rec_xyz.assign(geom->rec_xyz, geom->rec_xyz + 3 * ctx->total_rec);
    if (g.ndim == 2) {
        ctx->ntx = (g.nx + TX2 - 1) / TX2;
        ctx->ntz = (g.nz + TZ2 - 1) / TZ2;
        ctx->nty = 1;
        ctx->nzc = 1;
        ctx->ntiles = ctx->ntx * ctx->ntz;
    } else {
        ctx->ntx = (g.nx + TX3 - 1) / TX3;
        ctx->nty = (g.ny + TY3 - 1) / TY3;
        ctx->nzc = step3_chunks(g.nz, (long long)ctx->ntx * ctx->nty * geom->ns, ctx->esz);
        ctx->ntz = ctx->nzc;
        ctx->ntiles = ctx->ntx * ctx->nty * ctx->nzc;
    }
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) total_b = 0;
        ctx->dft_k = dft_block_steps((long long)ctx->ns * ctx->sst * ctx->esz, total_b);
    }
    if (const char *ev = std::getenv("ESI_NO_GRAPHS")) ctx->use_graphs = ev[0] == '0';
    if (const char *ev = std::getenv("ESI_PDL")) ctx->pdl = ev[0] != '0';
    esi_ctx *c = ctx.get();
    {
        esi_ctx *ctx = c;  // for CK
        CK(ctx->cc.ensure(ctx->sst * ctx->esz));
    }
    esi_status e = DISPATCH(c, create_impl)(c, velocity_dev);
    if (e != ESI_OK) {
        g_create_error = c->err;  // readable through esi_last_error(NULL)
        return e;
    }
    *out = ctx.release();
    return ESI_OK;
}

ESI_API void esi_destroy(esi_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->st);
    delete ctx;
}

ESI_API esi_status esi_set_stream(esi_ctx *ctx, void *stream) {
    if (!ctx) return ESI_ERR_ARG;
    ctx->st = reinterpret_cast<cudaStream_t>(stream);
    return ESI_OK;
}


ESI_API esi_status esi_set_shot_groups(esi_ctx *ctx, int groups, const void *velocity_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (groups < 1 || groups > ctx->ns)
        return ctx->fail(ESI_ERR_ARG, "groups must lie in 1 .. the number of shots");
    if (groups > 1 && !velocity_dev) return ctx->fail(ESI_ERR_ARG, "velocity_dev is NULL");
    ctx->err.clear();
    CK(cudaStreamSynchronize(ctx->st));
    ctx->clear_groups();
    if (groups == 1) return ESI_OK;
    esi_grid g = ctx->g;
    g.sponge_vref = ctx->vref;   // the groups' sponges take the context's reference velocity
    for (int k = 0; k < groups; ++k) {
        const int s0 = (int)((long long)k * ctx->ns / groups);
        const int s1 = (int)((long long)(k + 1) * ctx->ns / groups);
        std::vector<long long> off(s1 - s0 + 1);
        for (int s = s0; s <= s1; ++s) off[s - s0] = ctx->rec_off[s] - ctx->rec_off[s0];
        esi_geometry sub;
        sub.ns = s1 - s0;
        sub.src_xyz = ctx->src_xyz.data() + 3 * (size_t)s0;
        sub.rec_offset = off.data();
        sub.rec_xyz = ctx->rec_xyz.data() + 3 * (size_t)ctx->rec_off[s0];
        cudaStream_t st = nullptr;
        cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            ctx->clear_groups();
            return ctx->fail(ESI_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(ce));
        }
        ctx->grp_st.push_back(st);
        esi_ctx *c = nullptr;
        const esi_status e = esi_create(&c, &g, &sub, velocity_dev, ctx->dt, ctx->nt, st);
        if (e != ESI_OK) {
            const std::string m = esi_last_error(nullptr);
            ctx->clear_groups();
            return ctx->fail(e, "shot group " + std::to_string(k) + ": " + m);
        }
        c->use_graphs = ctx->use_graphs;
        c->pdl = ctx->pdl;
        c->prof = ctx->prof;
        ctx->grp.push_back(c);
        ctx->grp_s0.push_back(s0);
    }
    ctx->grp_s0.push_back(ctx->ns);
    for (int k = 0; k <= groups; ++k) {
        cudaEvent_t ev = nullptr;
        cudaError_t ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (ce != cudaSuccess) {
            ctx->clear_groups();
            return ctx->fail(ESI_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
        }
        ctx->grp_ev.push_back(ev);
    }
    return ESI_OK;
}

ESI_API esi_status esi_set_velocity(esi_ctx *ctx, const void *velocity_dev) {
    if (!ctx || !velocity_dev) return ESI_ERR_ARG;
    const esi_status e = ctx->g.dtype == ESI_F64 ? setup_model<double>(ctx, velocity_dev, false)
                                                 : setup_model<float>(ctx, velocity_dev, false);
    if (e != ESI_OK || ctx->grp.empty()) return e;
    // the groups follow the caller's model, each in its own thread (each set-up synchronises)
    return run_groups(ctx, [&](int, esi_ctx *c) { return esi_set_velocity(c, velocity_dev); });
}

ESI_API esi_status esi_forward(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                               void *traces_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (!traces_dev) return ctx->fail(ESI_ERR_ARG, "traces_dev is NULL");
    ctx->err.clear();
    if (!ctx->grp.empty())
        return run_groups(ctx, [&](int k, esi_ctx *c) {
            const int s0 = ctx->grp_s0[k];
            return esi_forward(c, at(wavelet_dev, (size_t)s0 * ctx->nt * ctx->esz),
                               at(ext_src_dev, field_off(ctx, s0)), at(traces_dev, trace_off(ctx, s0)));
        });
    return ctx->g.dtype == ESI_F64
               ? forward_impl<double>(ctx, wavelet_dev, ext_src_dev, traces_dev, nullptr, 0, nullptr)
               : forward_impl<float>(ctx, wavelet_dev, ext_src_dev, traces_dev, nullptr, 0, nullptr);
}

ESI_API esi_status esi_forward_noalloc(esi_ctx *ctx, const void *wavelet_dev,
                                       const void *ext_src_dev, void *traces_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (!traces_dev) return ctx->fail(ESI_ERR_ARG, "traces_dev is NULL");
    ctx->err.clear();
    return ctx->g.dtype == ESI_F64
               ? forward_noalloc_impl<double>(ctx, wavelet_dev, ext_src_dev, traces_dev)
               : forward_noalloc_impl<float>(ctx, wavelet_dev, ext_src_dev, traces_dev);
}

ESI_API esi_status esi_adjoint(esi_ctx *ctx, const void *traces_dev, void *ext_out_dev,
                               void *wavelet_out_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (!traces_dev || (!ext_out_dev && !wavelet_out_dev))
        return ctx->fail(ESI_ERR_ARG, "need adjoint data and at least one output");
    ctx->err.clear();
    if (!ctx->grp.empty())
        return run_groups(ctx, [&](int k, esi_ctx *c) {
            const int s0 = ctx->grp_s0[k];
            return esi_adjoint(c, at(traces_dev, trace_off(ctx, s0)), at(ext_out_dev, field_off(ctx, s0)),
                               at(wavelet_out_dev, (size_t)s0 * ctx->nt * ctx->esz));
        });
    return ctx->g.dtype == ESI_F64 ? adjoint_impl<double>(ctx, traces_dev, ext_out_dev, wavelet_out_dev)
                                   : adjoint_impl<float>(ctx, traces_dev, ext_out_dev, wavelet_out_dev);
}

ESI_API esi_status esi_gradient(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                                const void *dobs_dev, const void *adj_src_dev,
                                const esi_grad_opts *opts, void *grad_dev, double *misfit) {
    if (!ctx) return ESI_ERR_ARG;
    if (!opts || !grad_dev) return ctx->fail(ESI_ERR_ARG, "need options and a gradient buffer");
    if (opts->param < ESI_PARAM_C || opts->param > ESI_PARAM_M ||
        opts->ckpt_kind < ESI_CKPT_F32 || opts->ckpt_kind > ESI_CKPT_BF16)
        return ctx->fail(ESI_ERR_ARG, "bad gradient options");
    ctx->err.clear();
    if (!ctx->grp.empty()) {
        // each group's gradient (the sum over its shots) into [G][N] scratch, then their sum
        const int G = (int)ctx->grp.size();
        const size_t gb = (size_t)ctx->N * ctx->esz;
        CK(ctx->grp_grad.ensure(G * gb));
        std::vector<double> mis(G, 0.0);
        const esi_status e = run_groups(ctx, [&](int k, esi_ctx *c) {
            const int s0 = ctx->grp_s0[k];
            return esi_gradient(c, at(wavelet_dev, (size_t)s0 * ctx->nt * ctx->esz),
                                at(ext_src_dev, field_off(ctx, s0)), at(dobs_dev, trace_off(ctx, s0)),
                                at(adj_src_dev, trace_off(ctx, s0)), opts,
                                at(ctx->grp_grad.p, k * gb), misfit ? &mis[k] : nullptr);
        });
        if (e != ESI_OK) return e;
        if (ctx->g.dtype == ESI_F64)
            CKL(launch_sum_parts<double>(reinterpret_cast<double *>(grad_dev), ctx->grp_grad.as<double>(),
                                         G, ctx->N, ctx->st));
        else
            CKL(launch_sum_parts<float>(reinterpret_cast<float *>(grad_dev), ctx->grp_grad.as<float>(), G,
                                        ctx->N, ctx->st));
        if (misfit) {
            double t = 0.0;
            for (double m : mis) t += m;
            *misfit = t;
        }
        return ESI_OK;
    }
    return ctx->g.dtype == ESI_F64
               ? gradient_impl<double>(ctx, wavelet_dev, ext_src_dev, dobs_dev, adj_src_dev, opts,
                                       grad_dev, misfit)
               : gradient_impl<float>(ctx, wavelet_dev, ext_src_dev, dobs_dev, adj_src_dev, opts,
                                      grad_dev, misfit);
}

ESI_API esi_status esi_dft_extract(esi_ctx *ctx, const void *wavelet_dev, const void *ext_src_dev,
                                   const double *freqs_hz, int nf, void *out_dev, int out_kind,
                                   float *scales_host, void *traces_dev) {
    if (!ctx) return ESI_ERR_ARG;
    ctx->err.clear();
    if (!ctx->grp.empty() && nf > 0) {
        const size_t cell = out_kind == ESI_DFT_C32_HALF ? 4 : 2 * (size_t)ctx->esz;
        return run_groups(ctx, [&](int k, esi_ctx *c) {
            const int s0 = ctx->grp_s0[k];
            return esi_dft_extract(c, at(wavelet_dev, (size_t)s0 * ctx->nt * ctx->esz),
                                   at(ext_src_dev, field_off(ctx, s0)), freqs_hz, nf,
                                   at(out_dev, (size_t)s0 * nf * ctx->N * cell), out_kind,
                                   scales_host ? scales_host + (size_t)s0 * nf : nullptr,
                                   at(traces_dev, trace_off(ctx, s0)));
        });
    }
    return ctx->g.dtype == ESI_F64
               ? dft_impl<double>(ctx, wavelet_dev, ext_src_dev, freqs_hz, nf, out_dev, out_kind,
                                  scales_host, traces_dev)
               : dft_impl<float>(ctx, wavelet_dev, ext_src_dev, freqs_hz, nf, out_dev, out_kind,
                                 scales_host, traces_dev);
}

ESI_API esi_status esi_invert(esi_ctx *ctx, const esi_invert_opts *opts, const void *wavelet_dev,
                              const void *dobs_dev, void *velocity_dev, void *grad_dev,
                              esi_invert_report *report) {
    if (!ctx) return ESI_ERR_ARG;
    if (!opts || !dobs_dev || !velocity_dev || !grad_dev)
        return ctx->fail(ESI_ERR_ARG, "bad outer-loop arguments");
    ctx->err.clear();
    return ctx->g.dtype == ESI_F64
               ? invert_impl<double>(ctx, opts, wavelet_dev, dobs_dev, velocity_dev, grad_dev, report)
               : invert_impl<float>(ctx, opts, wavelet_dev, dobs_dev, velocity_dev, grad_dev, report);
}

ESI_API esi_status esi_fdcg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                  const void *dobs_dev, const double *freqs_hz, int nf,
                                  int precond, void *qbar_out_dev, double eps,
                                  esi_cg_report *report) {
    if (!ctx) return ESI_ERR_ARG;
    if (!dobs_dev || !qbar_out_dev || !freqs_hz || !(lambda > 0) || !(tol >= 0))
        return ctx->fail(ESI_ERR_ARG, "bad frequency-domain CG arguments");
    ctx->err.clear();
    if (!ctx->grp.empty() && nf >= 1)
        return run_group_solves(ctx, report, [&](int k, esi_ctx *c, esi_cg_report *r) {
            const int s0 = ctx->grp_s0[k];
            return esi_fdcg_solve(c, lambda, tol, max_iter, at(dobs_dev, trace_off(ctx, s0)),
                                  freqs_hz, nf, precond,
                                  at(qbar_out_dev, (size_t)s0 * nf * ctx->N * 2 * ctx->esz), eps, r);
        });
    return ctx->g.dtype == ESI_F64
               ? fdcg_impl<double>(ctx, lambda, tol, max_iter, dobs_dev, freqs_hz, nf, precond,
                                   qbar_out_dev, eps, report)
               : fdcg_impl<float>(ctx, lambda, tol, max_iter, dobs_dev, freqs_hz, nf, precond,
                                  qbar_out_dev, eps, report);
}

ESI_API esi_status esi_dscg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                  const void *dobs_dev, void *q_out_dev, void *w_out_dev,
                                  double eps, esi_cg_report *report) {
    if (!ctx) return ESI_ERR_ARG;
    if (!dobs_dev || !q_out_dev || !(lambda > 0) || !(tol >= 0))
        return ctx->fail(ESI_ERR_ARG, "bad data-space CG arguments");
    ctx->err.clear();
    if (!ctx->grp.empty())
        return run_group_solves(ctx, report, [&](int k, esi_ctx *c, esi_cg_report *r) {
            const int s0 = ctx->grp_s0[k];
            return esi_dscg_solve(c, lambda, tol, max_iter, at(dobs_dev, trace_off(ctx, s0)),
                                  at(q_out_dev, field_off(ctx, s0)), at(w_out_dev, trace_off(ctx, s0)),
                                  eps, r);
        });
    return ctx->g.dtype == ESI_F64
               ? dscg_impl<double>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, w_out_dev, eps,
                                   report)
               : dscg_impl<float>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, w_out_dev, eps,
                                  report);
}

ESI_API esi_status esi_wri_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                 const void *wavelet_dev, const void *dobs_dev, void *q_out_dev,
                                 esi_cg_report *report) {
    if (!ctx) return ESI_ERR_ARG;
    if (!wavelet_dev || !dobs_dev || !q_out_dev || !(lambda >= 0) || !(tol >= 0))
        return ctx->fail(ESI_ERR_ARG, "bad WRI arguments");
    ctx->err.clear();
    if (!ctx->grp.empty())
        return run_group_solves(ctx, report, [&](int k, esi_ctx *c, esi_cg_report *r) {
            const int s0 = ctx->grp_s0[k];
            return esi_wri_solve(c, lambda, tol, max_iter, at(wavelet_dev, (size_t)s0 * ctx->nt * ctx->esz),
                                 at(dobs_dev, trace_off(ctx, s0)), at(q_out_dev, field_off(ctx, s0)), r);
        });
    return ctx->g.dtype == ESI_F64
               ? cg_impl<double>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, ESI_PC_NONE, 0.0,
                                 report, wavelet_dev)
               : cg_impl<float>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, ESI_PC_NONE, 0.0,
                                report, wavelet_dev);
}

ESI_API esi_status esi_cg_solve(esi_ctx *ctx, double lambda, double tol, int max_iter,
                                const void *dobs_dev, void *q_out_dev, int precond, double eps,
                                esi_cg_report *report) {
    if (!ctx) return ESI_ERR_ARG;
    if (!dobs_dev || !q_out_dev || !(lambda >= 0) || !(tol >= 0))
        return ctx->fail(ESI_ERR_ARG, "bad CG arguments");
    ctx->err.clear();
    if (!ctx->grp.empty() && precond != ESI_PC_LEARNED) {
        // the network's buffers belong to this context: the learned solve runs here
        return run_group_solves(ctx, report, [&](int k, esi_ctx *c, esi_cg_report *r) {
            const int s0 = ctx->grp_s0[k];
            return esi_cg_solve(c, lambda, tol, max_iter, at(dobs_dev, trace_off(ctx, s0)),
                                at(q_out_dev, field_off(ctx, s0)), precond, eps, r);
        });
    }
    return ctx->g.dtype == ESI_F64
               ? cg_impl<double>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, precond, eps, report)
               : cg_impl<float>(ctx, lambda, tol, max_iter, dobs_dev, q_out_dev, precond, eps, report);
}

ESI_API esi_status esi_pc_load(esi_ctx *ctx, const void *weights_dev, size_t bytes) {
    if (!ctx) return ESI_ERR_ARG;
    if (!weights_dev || bytes != (size_t)pcnet::param_count() * sizeof(float))
        return ctx->fail(ESI_ERR_ARG, "weights must be esi_pc_param_count() FP32 values");
    if (ctx->g.ndim != 2 || ctx->g.dtype != ESI_F32)
        return ctx->fail(ESI_ERR_UNSUPPORTED, "the learned preconditioner serves 2D FP32 contexts");
    if (!ctx->pc) {
        const long long nimg = (long long)ctx->ns * ((ctx->nt + 15) / 16);
        ctx->pc_batch = (int)std::min<long long>(nimg, 512);
        std::string err;
        ctx->pc = pcnet_create((ctx->g.nz + 1) / 2, (ctx->g.nx + 1) / 2, ctx->pc_batch, ctx->st, &err);
        if (!ctx->pc) return ctx->fail(ESI_ERR_OOM, err);
    }
    CK(pcnet_set_params(ctx->pc, reinterpret_cast<const float *>(weights_dev), ctx->st));
    return ESI_OK;
}

ESI_API long long esi_pc_fallbacks(const esi_ctx *ctx) { return ctx ? ctx->pc_fallbacks : 0; }

ESI_API esi_status esi_normal_apply(esi_ctx *ctx, double lambda, double eps, const void *p_dev,
                                    void *out_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (!p_dev || !out_dev || !(lambda >= 0)) return ctx->fail(ESI_ERR_ARG, "bad arguments");
    ctx->err.clear();
    if (!ctx->grp.empty())
        return run_groups(ctx, [&](int k, esi_ctx *c) {
            const int s0 = ctx->grp_s0[k];
            return esi_normal_apply(c, lambda, eps, at(p_dev, field_off(ctx, s0)),
                                    at(out_dev, field_off(ctx, s0)));
        });
    CK(ctx->traces.ensure(std::max<size_t>((size_t)ctx->total_rec * ctx->nt * ctx->esz, 16)));
    const double ep = eps > 0 ? eps : ctx->g.dx;
    esi_status e;
    if (ctx->g.dtype == ESI_F64) {
        e = forward_impl<double>(ctx, nullptr, p_dev, ctx->traces.p, nullptr, 0, nullptr);
        if (e == ESI_OK) e = adjoint_impl<double>(ctx, ctx->traces.p, out_dev, nullptr);
        if (e == ESI_OK)
            CKL(launch_add_b2p<double>((double *)out_dev, (const double *)p_dev, ctx->ns, ctx->nt,
                                       ctx->g.nz, ctx->g.ny, ctx->g.nx, lambda, ep, ctx->g.dx,
                                       ctx->src_pos.as<double>(), ctx->st));
    } else {
        e = forward_impl<float>(ctx, nullptr, p_dev, ctx->traces.p, nullptr, 0, nullptr);
        if (e == ESI_OK) e = adjoint_impl<float>(ctx, ctx->traces.p, out_dev, nullptr);
        if (e == ESI_OK)
            CKL(launch_add_b2p<float>((float *)out_dev, (const float *)p_dev, ctx->ns, ctx->nt,
                                      ctx->g.nz, ctx->g.ny, ctx->g.nx, float(lambda), float(ep),
                                      float(ctx->g.dx), ctx->src_pos.as<double>(), ctx->st));
    }
    return e;
}

ESI_API esi_status esi_pc_pack(esi_ctx *ctx, const void *field_dev, double lambda, double eps,
                               int scale, int pitched, void *img_dev) {
    if (!ctx) return ESI_ERR_ARG;
    if (!field_dev || !img_dev) return ctx->fail(ESI_ERR_ARG, "bad arguments");
    if (ctx->g.ndim != 2 || ctx->g.dtype != ESI_F32)
        return ctx->fail(ESI_ERR_UNSUPPORTED, "packing serves 2D FP32 contexts");
    if (scale && !(lambda > 0)) return ctx->fail(ESI_ERR_ARG, "scaling needs lambda > 0");
    float *ipb2 = nullptr;
    if (scale) {
        CK(ctx->pb2.ensure((size_t)ctx->ns * ctx->sst * 4));
        CK(ctx->ipb2.ensure((size_t)ctx->ns * ctx->sst * 4));
        CKL(launch_b2_maps<float>(ctx->pb2.as<float>(), ctx->ipb2.as<float>(), ctx->ns, ctx->g.nz,
                                  ctx->g.ny, ctx->g.nx, ctx->px, float(lambda),
                                  float(eps > 0 ? eps : ctx->g.dx), float(ctx->g.dx),
                                  ctx->src_pos.as<double>(), 0, ctx->st));
        ipb2 = ctx->ipb2.as<float>();
    }
    CKL(pcnet::pack_launch(reinterpret_cast<const float *>(field_dev), ipb2,
                           reinterpret_cast<__nv_bfloat16 *>(img_dev), ctx->ns, ctx->nt, ctx->g.nz,
                           ctx->g.nx, ctx->px, ctx->sst, scale, pitched ? 0 : 1, ctx->st));
    return ESI_OK;
}

}  // extern "C"
