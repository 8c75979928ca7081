// nn.cuh -- argument structs and kernel declarations of the neural-operator
// layers (defined in nn.cu, launched by nop.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbib {
namespace nn {

struct ConvArgs {
    const __nv_bfloat16* in1;  // (N, H, W, C1)
    const __nv_bfloat16* in2;  // (N, H/2, W/2, C2) read upsampled, or NULL
    const __nv_bfloat16* w;    // (9, Co, Ci): tap, output channel, input channel
    const float* bias;         // (Co) or NULL
    void* out;                 // (N, H, W, Co) bf16, or fp32 when out_f32
    const __nv_bfloat16* gate; // (N, H, W, Co) or NULL: out = 0 where !(gate > 0) (ReLU backward)
    int N, H, W, C1, C2, Co;
    int relu, out_f32;
};

struct WgradArgs {
    const __nv_bfloat16* in1;
    const __nv_bfloat16* in2;
    const __nv_bfloat16* g;  // (N, H, W, Co)
    float* dw;               // (9, Ci, Co) FP32, accumulated
    float* db;               // (Co) FP32, accumulated, or NULL
    int N, H, W, C1, C2, Co;
    int tiles_per_cta;
};

constexpr int kTH = 8, kTW = 16;  // pixel tile of a CTA
constexpr int kConvSmem = (10 * 18 * 40 + 9 * 64 * 40) * 2;
constexpr int kWgSmem = 10 * 18 * 40 * 2 + 128 * 72 * 2;

__global__ void conv3x3_fwd_kernel(ConvArgs a);
__global__ void conv3x3_wgrad_kernel(WgradArgs a);
__global__ void avgpool2_kernel(const __nv_bfloat16* x, __nv_bfloat16* y, int N, int H, int W,
                                int C);
__global__ void avgpool2_bwd_kernel(const __nv_bfloat16* g, __nv_bfloat16* gx, int N, int H,
                                    int W, int C);
__global__ void concat_bwd_kernel(const __nv_bfloat16* g, __nv_bfloat16* gskip,
                                  __nv_bfloat16* gx2, const __nv_bfloat16* gate2, int N, int H,
                                  int W, int C1, int C2, int accumulate_skip);
__global__ void add_gate_kernel(__nv_bfloat16* g, const __nv_bfloat16* h,
                                const __nv_bfloat16* act, int64_t n);
__global__ void mse_kernel(const float* y, int Cy, const float* t, __nv_bfloat16* dy, int Cdy,
                           int64_t n, double* loss);
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2);
__global__ void weight_copies_kernel(const float* w, int Ci, int Co, int Cip, int Cop,
                                     __nv_bfloat16* wf, __nv_bfloat16* wd);
__global__ void features_kernel(const uint8_t* id_mask, const uint8_t* src, const float* Dn,
                                const float* Kn, __nv_bfloat16* x, int N, int HW);
__global__ void scale_kernel(const float* in, int Cin, float* out, const float* fac, int N,
                             int HW);

}  // namespace nn

// The tcgen05 convolution (conv_tc.cu): whether a layer's shape is supported
// (W up to 128 or a multiple of 128, channels multiples of 16, C1 a multiple
// of the chunk width), the element count of its tiled weights, the tiling of
// (9, Co, Ci) weights, and the convolution itself (out as nn::ConvArgs, the
// tiled weights in place of c.w; err raised when a bounded wait ran out).
bool tc_conv_supported(int H, int W, int C1, int C2, int Co);
int64_t tc_tiled_weight_elems(int Ci, int Co);
cudaError_t tc_tile_weights(const void* w, int Co, int Ci, void* wt, cudaStream_t s);
cudaError_t tc_conv3x3(const nn::ConvArgs& c, const void* wt, unsigned* err, cudaStream_t s);
// The weight gradient on tcgen05 (conv_tc.cu): whether a layer's shape is
// supported (W from 16 up to 128 in multiples of 16, or a multiple of 128;
// channels multiples of 16, at most 384 input channels), and the
// gradient itself (w.dw and w.db accumulated; err as for the convolution).
bool tc_wgrad_supported(int H, int W, int C1, int C2, int Co);
cudaError_t tc_conv3x3_wgrad(const nn::WgradArgs& w, unsigned* err, cudaStream_t s);

// One layer of the fused weight refresh: the FP32 master weights w (9, Ci, Co)
// and the BF16 copies made from them -- the forward copy wf (9, Co, Ci), the
// tap-flipped data-gradient copy wd (9, Ci, Co) and the tcgen05 tilings of
// both (wft, wdt).
struct WeightSet {
    const float* w;
    __nv_bfloat16 *wf, *wd, *wft, *wdt;
    int Ci, Co;
};
// All layers' copies in one launch (d_sets: the table in device memory, n
// entries; max_elems: the largest per-layer element count, for the grid).
cudaError_t refresh_weight_sets(const WeightSet* d_sets, int n, int64_t max_elems, cudaStream_t s);
int64_t weight_set_elems(int Ci, int Co);
}  // namespace lbib
