// Internal declarations of the learned preconditioner (U-Net on time-grouped images).
#pragma once

#include <cuda_bf16.h>

#include "esi_internal.h"

namespace esi {

// cuTensorMapEncodeTiled obtained through the runtime (defined in esi_api.cu)
using TensorMapEncoder = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                      const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                      const cuuint32_t *, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion,
                                      CUtensorMapFloatOOBfill);
TensorMapEncoder tensor_map_encoder();

namespace pcnet {

constexpr int G = 16;   // time samples per image = network input / output channels
constexpr int C = 32;   // hidden channels
constexpr int NLAYER = 7;

struct LayerDef {
    int cin, cout;
    bool relu;
};
// enc1, enc2, enc3, bott, dec3, dec2, dec1 (parameter order: W[3][3][cin][cout], b[cout])
constexpr LayerDef LAYERS[NLAYER] = {{G, C, true},  {C, C, true}, {C, C, true}, {C, C, true},
                                     {C, C, true},  {C, C, true}, {C, G, false}};

constexpr long long layer_params(int l) {
    return 9ll * LAYERS[l].cin * LAYERS[l].cout + LAYERS[l].cout;
}
constexpr long long param_count() {
    long long n = 0;
    for (int l = 0; l < NLAYER; ++l) n += layer_params(l);
    return n;
}

// activation map [n][H][W][C_] BF16, box (8 channels, 130 columns, 1 row, 1 image)
cudaError_t make_act_map(CUtensorMap *tm, const void *base, int C_, int W, int H, int n);
// conv epilogue options
struct ConvEpi {
    const float *oscale = nullptr;   // per-image output factor (applied after the activation)
    const float *irms = nullptr;     // per-image input RMS: the accumulator is divided by it
    int nchw = 0;                    // output planes [img][c][H][W] instead of channels-last
};
template <int CIN, int COUT, bool RELU, typename OUT>
cudaError_t conv_launch(const void *in, const __nv_bfloat16 *wprep, const float *bias, OUT *out,
                        int nimg, int H, int W, int *dev_err, int nsm, cudaStream_t st,
                        const ConvEpi &epi = ConvEpi());
// rms[i] = root-mean-square of image i (acc: n FP64 scratch sums); xn = x / rms (BF16)
// unless xn is null
cudaError_t normalize_launch(const __nv_bfloat16 *x, float *rms, double *acc, __nv_bfloat16 *xn,
                             int n, long long per, cudaStream_t st);
cudaError_t img_mul_launch(float *g, const float *s, int n, long long per, cudaStream_t st);
cudaError_t wprep_launch(const float *W, __nv_bfloat16 *out, int cin, int cout, int flip,
                         cudaStream_t st);
cudaError_t pack_launch(const float *r, const float *ipb2, __nv_bfloat16 *img, int ns, int nt,
                        int nz, int nx, int px, long long sst, int scale_by_map, int dense,
                        cudaStream_t st);
cudaError_t pool_launch(const __nv_bfloat16 *in, __nv_bfloat16 *out, long long n, int H, int W,
                        cudaStream_t st);
cudaError_t upadd_launch(const __nv_bfloat16 *coarse, const __nv_bfloat16 *skip,
                         __nv_bfloat16 *out, long long n, int H, int W, cudaStream_t st);
cudaError_t mask_launch(float *g, const __nv_bfloat16 *act, __nv_bfloat16 *gb, long long n,
                        cudaStream_t st);
cudaError_t pool_bwd_launch(float *gf, const float *gc, long long n, int H, int W, cudaStream_t st);
cudaError_t up_bwd_launch(const float *gf, float *gc, long long n, int H, int W, cudaStream_t st);
template <int CIN, int COUT>
cudaError_t dw_launch(const __nv_bfloat16 *x, const __nv_bfloat16 *gy, float *part, float *gW,
                      int nimg, int H, int W, int nblk, cudaStream_t st);
cudaError_t bias_grad_launch(const float *g, float *gb, long long npix, int Cn, cudaStream_t st);
cudaError_t cos_loss_launch(const __nv_bfloat16 *in, const float *y, const __nv_bfloat16 *e,
                            double *dots, float *gy, long long per, int nimg, cudaStream_t st);
cudaError_t adam_launch(float *p, const float *g, float *m, float *v, long long n, float lr, int t,
                        cudaStream_t st);
// per-shot partial sums of <s, r>, <y, r>, <s, ap>, <y, ap> (s = r ipb2, y = the network's
// time-sample planes upsampled 2 x 2) into part[4][ns][nblk]; ap may be null
cudaError_t pc_dots_launch(const float *r, const float *ap, const float *ipb2, const float *y,
                           double *part, int nblk, int ns, int nt, int nz, int nx, int px,
                           long long sst, const int *active, cudaStream_t st);

}  // namespace pcnet

// The network object used by the C ABI and by the preconditioned CG.
struct PcNet;
PcNet *pcnet_create(int H1, int W1, int max_batch, cudaStream_t st, std::string *err);
void pcnet_destroy(PcNet *p);
cudaError_t pcnet_set_params(PcNet *p, const float *params_dev, cudaStream_t st);
cudaError_t pcnet_get_params(const PcNet *p, float *params_dev, cudaStream_t st);
// y = rms(x) U(x / rms(x)) per image (positively homogeneous in x, as a preconditioner must
// be): y[n][H1][W1][G] (FP32) for x[n][H1][W1][G] (BF16); n <= max_batch per call.  With
// nchw the output is y[n][G][H1][W1] (time-sample planes); with keep_xn the normalised input
// is materialised (BF16) for the weight gradient of the first layer, else the first layer
// divides its accumulator by rms.
cudaError_t pcnet_forward(PcNet *p, const __nv_bfloat16 *x, int n, float *y, cudaStream_t st,
                          bool nchw = false, bool keep_xn = false);
// loss = mean over images of 1 - cos^2(x + y, e); gradient of it into p's gradient buffer;
// optional copy of the gradient to grad_out (FP32, parameter layout)
cudaError_t pcnet_grad(PcNet *p, const __nv_bfloat16 *x, const __nv_bfloat16 *e, int n,
                       double *loss, float *grad_out, cudaStream_t st);
// parameter gradient of <gy, y(x)> for an output gradient gy (channels-last FP32)
cudaError_t pcnet_vjp(PcNet *p, const __nv_bfloat16 *x, const float *gy, int n, float *grad_out,
                      cudaStream_t st);
cudaError_t pcnet_adam(PcNet *p, double lr, cudaStream_t st);
int *pcnet_dev_err(PcNet *p);

}  // namespace esi
