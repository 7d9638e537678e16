// Host side of the learned preconditioner: the network object (FP32 master parameters,
// BF16 tensor-core weight copies, Adam moments, per-level activation and gradient buffers),
// its forward / backward orchestration, and the esi_pc_* C ABI.
#include <cmath>
#include <string>
#include <vector>

#include "esi_pc.h"

namespace esi {
namespace {

struct Buf {
    void *p = nullptr;
    size_t n = 0;
    ~Buf() {
        if (p) cudaFree(p);
    }
    cudaError_t ensure(size_t b) {
        if (p && b <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, b ? b : 16);
        if (e == cudaSuccess) n = b;
        return e;
    }
    template <typename U>
    U *as() const { return reinterpret_cast<U *>(p); }
};

}  // namespace

struct PcNet {
    int H[4], W[4];     // level sizes (level 0 = input resolution)
    int max_batch = 0;
    int nsm = 148;
    long long off[pcnet::NLAYER];   // parameter offsets (W then b) of each layer
    Buf params, grads, m, v, wf, wb;   // wf / wb: BF16 forward / flipped weights per layer
    long long wf_off[pcnet::NLAYER];
    int adam_t = 0;
    // activations (BF16, 32 channels unless noted)
    Buf e1, p1, e2, p2, e3, p3, bt, u3, d3, u2, d2, u1;
    // gradients (FP32) and BF16 staging
    Buf gy, gL1, gD2, gL2, gD3, gL3, gBT, gP3, gP2, gP1, gbf, dwpart, yscratch, dots;
    Buf xn, rms;    // normalised input images and their per-image scale
    Buf rms_acc;    // per-image FP64 sums of squares
    Buf dev_err;
    bool weights_ready = false;
};

namespace {

using namespace pcnet;

long long px_of(const PcNet *p, int l, int n) { return (long long)n * p->H[l] * p->W[l]; }

cudaError_t prep_weights(PcNet *p, cudaStream_t st) {
    for (int l = 0; l < NLAYER; ++l) {
        const int ci = LAYERS[l].cin, co = LAYERS[l].cout;
        const float *W = p->params.as<float>() + p->off[l];
        cudaError_t e = wprep_launch(W, p->wf.as<__nv_bfloat16>() + p->wf_off[l], ci, co, 0, st);
        if (e != cudaSuccess) return e;
        e = wprep_launch(W, p->wb.as<__nv_bfloat16>() + p->wf_off[l], ci, co, 1, st);
        if (e != cudaSuccess) return e;
    }
    p->weights_ready = true;
    return cudaSuccess;
}

const float *bias_of(const PcNet *p, int l) {
    return p->params.as<float>() + p->off[l] + 9ll * LAYERS[l].cin * LAYERS[l].cout;
}

#define RET(x)                              \
    do {                                    \
        cudaError_t _e = (x);               \
        if (_e != cudaSuccess) return _e;   \
    } while (0)

}  // namespace

PcNet *pcnet_create(int H1, int W1, int max_batch, cudaStream_t st, std::string *err) {
    if (H1 < 1 || W1 < 1 || max_batch < 1) {
        *err = "bad preconditioner size";
        return nullptr;
    }
    PcNet *p = new PcNet();
    p->max_batch = max_batch;
    p->H[0] = H1;
    p->W[0] = W1;
    for (int l = 1; l < 4; ++l) {
        p->H[l] = (p->H[l - 1] + 1) / 2;
        p->W[l] = (p->W[l - 1] + 1) / 2;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
    long long o = 0, wo = 0;
    for (int l = 0; l < NLAYER; ++l) {
        p->off[l] = o;
        o += layer_params(l);
        p->wf_off[l] = wo;
        wo += 9ll * LAYERS[l].cin * LAYERS[l].cout;
    }
    const size_t np = (size_t)param_count() * sizeof(float);
    const int n = max_batch;
    auto act = [&](Buf &b, int l, int ch) { return b.ensure((size_t)px_of(p, l, n) * ch * 2); };
    cudaError_t e = cudaSuccess;
    if ((e = p->params.ensure(np)) || (e = p->grads.ensure(np)) || (e = p->m.ensure(np)) ||
        (e = p->v.ensure(np)) || (e = p->wf.ensure(wo * 2)) || (e = p->wb.ensure(wo * 2)) ||
        (e = act(p->e1, 0, C)) || (e = act(p->p1, 1, C)) || (e = act(p->e2, 1, C)) ||
        (e = act(p->p2, 2, C)) || (e = act(p->e3, 2, C)) || (e = act(p->p3, 3, C)) ||
        (e = act(p->bt, 3, C)) || (e = act(p->u3, 2, C)) || (e = act(p->d3, 2, C)) ||
        (e = act(p->u2, 1, C)) || (e = act(p->d2, 1, C)) || (e = act(p->u1, 0, C)) ||
        (e = p->dev_err.ensure(sizeof(int))) || (e = p->dots.ensure(sizeof(double) * 3 * n)) ||
        (e = act(p->xn, 0, G)) || (e = p->rms.ensure(sizeof(float) * n)) ||
        (e = p->rms_acc.ensure(sizeof(double) * n))) {
        *err = std::string("preconditioner allocation: ") + cudaGetErrorString(e);
        delete p;
        return nullptr;
    }
    cudaMemsetAsync(p->params.p, 0, np, st);
    cudaMemsetAsync(p->m.p, 0, np, st);
    cudaMemsetAsync(p->v.p, 0, np, st);
    cudaMemsetAsync(p->dev_err.p, 0, sizeof(int), st);
    return p;
}

void pcnet_destroy(PcNet *p) { delete p; }

int *pcnet_dev_err(PcNet *p) { return p->dev_err.as<int>(); }

cudaError_t pcnet_set_params(PcNet *p, const float *src, cudaStream_t st) {
    RET(cudaMemcpyAsync(p->params.p, src, (size_t)param_count() * 4, cudaMemcpyDeviceToDevice, st));
    RET(cudaMemsetAsync(p->m.p, 0, p->m.n, st));
    RET(cudaMemsetAsync(p->v.p, 0, p->v.n, st));
    p->adam_t = 0;
    return prep_weights(p, st);
}

cudaError_t pcnet_get_params(const PcNet *p, float *dst, cudaStream_t st) {
    return cudaMemcpyAsync(dst, p->params.p, (size_t)param_count() * 4, cudaMemcpyDeviceToDevice, st);
}

cudaError_t pcnet_forward(PcNet *p, const __nv_bfloat16 *x, int n, float *y, cudaStream_t st,
                          bool nchw, bool keep_xn) {
    if (n > p->max_batch || n < 1) return cudaErrorInvalidValue;
    if (!p->weights_ready) RET(prep_weights(p, st));
    const int *H = p->H, *W = p->W;
    int *de = p->dev_err.as<int>();
    auto wf = [&](int l) { return p->wf.as<__nv_bfloat16>() + p->wf_off[l]; };
    using bf = __nv_bfloat16;
    RET(normalize_launch(x, p->rms.as<float>(), p->rms_acc.as<double>(), keep_xn ? p->xn.as<bf>() : nullptr, n,
                         (long long)H[0] * W[0] * G, st));
    ConvEpi e0;
    if (keep_xn)
        x = p->xn.as<bf>();
    else
        e0.irms = p->rms.as<float>();   // conv(x / rms) = conv(x) / rms before the bias
    RET((conv_launch<G, C, true, bf>(x, wf(0), bias_of(p, 0), p->e1.as<bf>(), n, H[0], W[0], de, p->nsm, st, e0)));
    RET(pool_launch(p->e1.as<bf>(), p->p1.as<bf>(), n, H[0], W[0], st));
    RET((conv_launch<C, C, true, bf>(p->p1.p, wf(1), bias_of(p, 1), p->e2.as<bf>(), n, H[1], W[1], de, p->nsm, st)));
    RET(pool_launch(p->e2.as<bf>(), p->p2.as<bf>(), n, H[1], W[1], st));
    RET((conv_launch<C, C, true, bf>(p->p2.p, wf(2), bias_of(p, 2), p->e3.as<bf>(), n, H[2], W[2], de, p->nsm, st)));
    RET(pool_launch(p->e3.as<bf>(), p->p3.as<bf>(), n, H[2], W[2], st));
    RET((conv_launch<C, C, true, bf>(p->p3.p, wf(3), bias_of(p, 3), p->bt.as<bf>(), n, H[3], W[3], de, p->nsm, st)));
    RET(upadd_launch(p->bt.as<bf>(), p->e3.as<bf>(), p->u3.as<bf>(), n, H[2], W[2], st));
    RET((conv_launch<C, C, true, bf>(p->u3.p, wf(4), bias_of(p, 4), p->d3.as<bf>(), n, H[2], W[2], de, p->nsm, st)));
    RET(upadd_launch(p->d3.as<bf>(), p->e2.as<bf>(), p->u2.as<bf>(), n, H[1], W[1], st));
    RET((conv_launch<C, C, true, bf>(p->u2.p, wf(5), bias_of(p, 5), p->d2.as<bf>(), n, H[1], W[1], de, p->nsm, st)));
    RET(upadd_launch(p->d2.as<bf>(), p->e1.as<bf>(), p->u1.as<bf>(), n, H[0], W[0], st));
    ConvEpi e6;
    e6.oscale = p->rms.as<float>();
    e6.nchw = nchw ? 1 : 0;
    RET((conv_launch<C, G, false, float>(p->u1.p, wf(6), bias_of(p, 6), y, n, H[0], W[0], de, p->nsm, st, e6)));
    return cudaSuccess;
}

namespace {

// scratch of the backward pass for n images
cudaError_t ensure_grad_buffers(PcNet *p, int n) {
    const long long n0 = px_of(p, 0, n), n1 = px_of(p, 1, n), n2 = px_of(p, 2, n), n3 = px_of(p, 3, n);
    RET(p->yscratch.ensure((size_t)n0 * G * 4));
    RET(p->gy.ensure((size_t)n0 * G * 4));
    RET(p->gL1.ensure((size_t)n0 * C * 4));
    RET(p->gD2.ensure((size_t)n1 * C * 4));
    RET(p->gL2.ensure((size_t)n1 * C * 4));
    RET(p->gP1.ensure((size_t)n1 * C * 4));
    RET(p->gD3.ensure((size_t)n2 * C * 4));
    RET(p->gL3.ensure((size_t)n2 * C * 4));
    RET(p->gP2.ensure((size_t)n2 * C * 4));
    RET(p->gBT.ensure((size_t)n3 * C * 4));
    RET(p->gP3.ensure((size_t)n3 * C * 4));
    RET(p->gbf.ensure((size_t)n0 * C * 2));
    RET(p->dwpart.ensure((size_t)9 * 2 * p->nsm * C * C * 4));
    return cudaSuccess;
}

// Parameter gradient of <gy, y(x)> into p->grads (overwritten), gy = dL/dy in p->gy
// (channels-last FP32), after pcnet_forward(x, keep_xn = true) of the same n images.
cudaError_t backward_from_gy(PcNet *p, int n, cudaStream_t st) {
    using bf = __nv_bfloat16;
    const int *H = p->H, *W = p->W;
    const long long n0 = px_of(p, 0, n), n1 = px_of(p, 1, n), n2 = px_of(p, 2, n), n3 = px_of(p, 3, n);
    const int nblk = 2 * p->nsm;
    // y = rms * U(xn): the network's output gradient carries the per-image scale
    RET(img_mul_launch(p->gy.as<float>(), p->rms.as<float>(), n, (long long)H[0] * W[0] * G, st));
    const bf *xin = p->xn.as<bf>();   // the first layer saw the normalised images
    int *de = p->dev_err.as<int>();
    auto wb = [&](int l) { return p->wb.as<__nv_bfloat16>() + p->wf_off[l]; };
    auto gW = [&](int l) { return p->grads.as<float>() + p->off[l]; };
    auto gB = [&](int l) { return p->grads.as<float>() + p->off[l] + 9ll * LAYERS[l].cin * LAYERS[l].cout; };
    bf *gb = p->gbf.as<bf>();
    float *dw = p->dwpart.as<float>();
    // dec1 (linear): input u1, output y
    RET(mask_launch(p->gy.as<float>(), nullptr, gb, n0 * G, st));
    RET((dw_launch<C, G>(p->u1.as<bf>(), gb, dw, gW(6), n, H[0], W[0], nblk, st)));
    RET(bias_grad_launch(p->gy.as<float>(), gB(6), n0, G, st));
    RET((conv_launch<G, C, false, float>(gb, wb(6), nullptr, p->gL1.as<float>(), n, H[0], W[0], de, p->nsm, st)));
    // u1 = up(d2) + e1: e1 collects gL1 (in place); d2 gets up_bwd(gL1)
    RET(up_bwd_launch(p->gL1.as<float>(), p->gD2.as<float>(), n, H[0], W[0], st));
    // dec2: input u2, output d2 (ReLU)
    RET(mask_launch(p->gD2.as<float>(), p->d2.as<bf>(), gb, n1 * C, st));
    RET((dw_launch<C, C>(p->u2.as<bf>(), gb, dw, gW(5), n, H[1], W[1], nblk, st)));
    RET(bias_grad_launch(p->gD2.as<float>(), gB(5), n1, C, st));
    RET((conv_launch<C, C, false, float>(gb, wb(5), nullptr, p->gL2.as<float>(), n, H[1], W[1], de, p->nsm, st)));
    RET(up_bwd_launch(p->gL2.as<float>(), p->gD3.as<float>(), n, H[1], W[1], st));
    // dec3: input u3, output d3
    RET(mask_launch(p->gD3.as<float>(), p->d3.as<bf>(), gb, n2 * C, st));
    RET((dw_launch<C, C>(p->u3.as<bf>(), gb, dw, gW(4), n, H[2], W[2], nblk, st)));
    RET(bias_grad_launch(p->gD3.as<float>(), gB(4), n2, C, st));
    RET((conv_launch<C, C, false, float>(gb, wb(4), nullptr, p->gL3.as<float>(), n, H[2], W[2], de, p->nsm, st)));
    RET(up_bwd_launch(p->gL3.as<float>(), p->gBT.as<float>(), n, H[2], W[2], st));
    // bott: input p3, output bt
    RET(mask_launch(p->gBT.as<float>(), p->bt.as<bf>(), gb, n3 * C, st));
    RET((dw_launch<C, C>(p->p3.as<bf>(), gb, dw, gW(3), n, H[3], W[3], nblk, st)));
    RET(bias_grad_launch(p->gBT.as<float>(), gB(3), n3, C, st));
    RET((conv_launch<C, C, false, float>(gb, wb(3), nullptr, p->gP3.as<float>(), n, H[3], W[3], de, p->nsm, st)));
    RET(pool_bwd_launch(p->gL3.as<float>(), p->gP3.as<float>(), n, H[2], W[2], st));   // e3 grad
    // enc3: input p2, output e3
    RET(mask_launch(p->gL3.as<float>(), p->e3.as<bf>(), gb, n2 * C, st));
    RET((dw_launch<C, C>(p->p2.as<bf>(), gb, dw, gW(2), n, H[2], W[2], nblk, st)));
    RET(bias_grad_launch(p->gL3.as<float>(), gB(2), n2, C, st));
    RET((conv_launch<C, C, false, float>(gb, wb(2), nullptr, p->gP2.as<float>(), n, H[2], W[2], de, p->nsm, st)));
    RET(pool_bwd_launch(p->gL2.as<float>(), p->gP2.as<float>(), n, H[1], W[1], st));   // e2 grad
    // enc2: input p1, output e2
    RET(mask_launch(p->gL2.as<float>(), p->e2.as<bf>(), gb, n1 * C, st));
    RET((dw_launch<C, C>(p->p1.as<bf>(), gb, dw, gW(1), n, H[1], W[1], nblk, st)));
    RET(bias_grad_launch(p->gL2.as<float>(), gB(1), n1, C, st));
    RET((conv_launch<C, C, false, float>(gb, wb(1), nullptr, p->gP1.as<float>(), n, H[1], W[1], de, p->nsm, st)));
    RET(pool_bwd_launch(p->gL1.as<float>(), p->gP1.as<float>(), n, H[0], W[0], st));   // e1 grad
    // enc1: input x, output e1
    RET(mask_launch(p->gL1.as<float>(), p->e1.as<bf>(), gb, n0 * C, st));
    RET((dw_launch<G, C>(xin, gb, dw, gW(0), n, H[0], W[0], nblk, st)));
    RET(bias_grad_launch(p->gL1.as<float>(), gB(0), n0, C, st));
    return cudaSuccess;
}

}  // namespace

cudaError_t pcnet_grad(PcNet *p, const __nv_bfloat16 *x, const __nv_bfloat16 *e, int n,
                       double *loss, float *grad_out, cudaStream_t st) {
    if (n > p->max_batch || n < 1) return cudaErrorInvalidValue;
    const int *H = p->H, *W = p->W;
    RET(ensure_grad_buffers(p, n));
    float *y = p->yscratch.as<float>();
    RET(pcnet_forward(p, x, n, y, st, false, true));
    RET(cos_loss_launch(x, y, e, p->dots.as<double>(), p->gy.as<float>(), (long long)H[0] * W[0] * G, n, st));
    RET(backward_from_gy(p, n, st));
    if (grad_out)
        RET(cudaMemcpyAsync(grad_out, p->grads.p, (size_t)param_count() * 4, cudaMemcpyDeviceToDevice, st));
    if (loss) {
        std::vector<double> d(3 * (size_t)n);
        RET(cudaMemcpyAsync(d.data(), p->dots.p, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
        RET(cudaStreamSynchronize(st));
        double s = 0;
        for (int i = 0; i < n; ++i) {
            const double ze = d[3 * i], zz = d[3 * i + 1], ee = d[3 * i + 2];
            s += (zz > 0 && ee > 0) ? 1.0 - ze * ze / (zz * ee) : 0.0;
        }
        *loss = s / n;
    }
    return cudaSuccess;
}

cudaError_t pcnet_vjp(PcNet *p, const __nv_bfloat16 *x, const float *gy, int n, float *grad_out,
                      cudaStream_t st) {
    if (n > p->max_batch || n < 1) return cudaErrorInvalidValue;
    RET(ensure_grad_buffers(p, n));
    RET(pcnet_forward(p, x, n, p->yscratch.as<float>(), st, false, true));
    RET(cudaMemcpyAsync(p->gy.p, gy, (size_t)px_of(p, 0, n) * G * 4, cudaMemcpyDeviceToDevice, st));
    RET(backward_from_gy(p, n, st));
    if (grad_out)
        RET(cudaMemcpyAsync(grad_out, p->grads.p, (size_t)param_count() * 4, cudaMemcpyDeviceToDevice, st));
    return cudaSuccess;
}

cudaError_t pcnet_adam(PcNet *p, double lr, cudaStream_t st) {
    ++p->adam_t;
    RET(adam_launch(p->params.as<float>(), p->grads.as<float>(), p->m.as<float>(), p->v.as<float>(),
                    param_count(), (float)lr, p->adam_t, st));
    return prep_weights(p, st);
}

}  // namespace esi

// ----------------------------------------------------------------------------- C ABI
struct esi_pc {
    esi::PcNet *net = nullptr;
    cudaStream_t st = nullptr;
    std::string err;
};

namespace {
thread_local std::string g_pc_create_error;

esi_status pc_fail(esi_pc *pc, cudaError_t e, const char *what) {
    pc->err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ESI_ERR_OOM : ESI_ERR_CUDA;
}

esi_status pc_check_err(esi_pc *pc) {
    int h = 0;
    cudaMemcpyAsync(&h, esi::pcnet_dev_err(pc->net), sizeof(int), cudaMemcpyDeviceToHost, pc->st);
    cudaError_t e = cudaStreamSynchronize(pc->st);
    if (e != cudaSuccess) return pc_fail(pc, e, "preconditioner");
    if (h) {
        pc->err = "a tensor-core tile wait ran out of its iteration limit";
        return ESI_ERR_TIMEOUT;
    }
    return ESI_OK;
}
}  // namespace

extern "C" {

ESI_API size_t esi_pc_param_count(void) { return (size_t)esi::pcnet::param_count(); }

ESI_API esi_status esi_pc_create(esi_pc **out, int h, int w, int max_batch, void *stream) {
    g_pc_create_error.clear();
    if (!out) return ESI_ERR_ARG;
    *out = nullptr;
    esi_pc *pc = new esi_pc();
    pc->st = reinterpret_cast<cudaStream_t>(stream);
    pc->net = esi::pcnet_create(h, w, max_batch, pc->st, &g_pc_create_error);
    if (!pc->net) {
        delete pc;
        return ESI_ERR_OOM;
    }
    *out = pc;
    return ESI_OK;
}

ESI_API void esi_pc_destroy(esi_pc *pc) {
    if (!pc) return;
    cudaStreamSynchronize(pc->st);
    esi::pcnet_destroy(pc->net);
    delete pc;
}

ESI_API const char *esi_pc_last_error(const esi_pc *pc) {
    return pc ? pc->err.c_str() : g_pc_create_error.c_str();
}

ESI_API esi_status esi_pc_set_params(esi_pc *pc, const float *params_dev) {
    if (!pc || !params_dev) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_set_params(pc->net, params_dev, pc->st);
    return e == cudaSuccess ? ESI_OK : pc_fail(pc, e, "set_params");
}

ESI_API esi_status esi_pc_get_params(esi_pc *pc, float *params_dev) {
    if (!pc || !params_dev) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_get_params(pc->net, params_dev, pc->st);
    return e == cudaSuccess ? ESI_OK : pc_fail(pc, e, "get_params");
}

ESI_API esi_status esi_pc_apply(esi_pc *pc, const void *in_dev, int n, float *y_dev) {
    if (!pc || !in_dev || !y_dev || n < 1) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_forward(pc->net, reinterpret_cast<const __nv_bfloat16 *>(in_dev), n,
                                       y_dev, pc->st);
    if (e != cudaSuccess) return pc_fail(pc, e, "apply");
    return ESI_OK;
}

ESI_API esi_status esi_pc_grad(esi_pc *pc, const void *in_dev, const void *target_dev, int n,
                               float *grad_dev, double *loss) {
    if (!pc || !in_dev || !target_dev || n < 1) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_grad(pc->net, reinterpret_cast<const __nv_bfloat16 *>(in_dev),
                                    reinterpret_cast<const __nv_bfloat16 *>(target_dev), n, loss,
                                    grad_dev, pc->st);
    if (e != cudaSuccess) return pc_fail(pc, e, "grad");
    return pc_check_err(pc);
}

ESI_API esi_status esi_pc_vjp(esi_pc *pc, const void *in_dev, const float *gy_dev, int n,
                              float *grad_dev) {
    if (!pc || !in_dev || !gy_dev || !grad_dev || n < 1) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_vjp(pc->net, reinterpret_cast<const __nv_bfloat16 *>(in_dev), gy_dev,
                                   n, grad_dev, pc->st);
    if (e != cudaSuccess) return pc_fail(pc, e, "vjp");
    return ESI_OK;
}

ESI_API esi_status esi_pc_train_step(esi_pc *pc, const void *in_dev, const void *target_dev, int n,
                                     double lr, double *loss) {
    if (!pc || !in_dev || !target_dev || n < 1 || !(lr > 0)) return ESI_ERR_ARG;
    cudaError_t e = esi::pcnet_grad(pc->net, reinterpret_cast<const __nv_bfloat16 *>(in_dev),
                                    reinterpret_cast<const __nv_bfloat16 *>(target_dev), n, loss,
                                    nullptr, pc->st);
    if (e == cudaSuccess) e = esi::pcnet_adam(pc->net, lr, pc->st);
    if (e != cudaSuccess) return pc_fail(pc, e, "train_step");
    return loss ? pc_check_err(pc) : ESI_OK;
}

}  // extern "C"
