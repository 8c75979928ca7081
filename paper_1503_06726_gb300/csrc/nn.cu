// nn.cu -- kernels of the neural operator that warm-starts the steady
// morphogen solve: BF16 tensor-core 3x3 convolutions (forward, data
// gradient, weight gradient) with FP32 accumulation, and the elementwise
// layers (pooling, ReLU gradient, loss, Adam).  NHWC activations in BF16,
// channel counts multiples of 16.
//
// Convolution as an implicit GEMM: M = output pixels (a CTA tile of 8 x 16
// pixels of one image), N = output channels (64 per CTA), K = 9 taps x input
// channels (chunks of 32).  Per K chunk the CTA stages the 10 x 18 halo of
// its pixel tile and the weights of all 9 taps in shared memory with
// cp.async (zero fill outside the image), then every warp multiplies its
// 32 x 32 block with mma.sync m16n8k16 (BF16 in, FP32 accumulate) fed by
// ldmatrix.  The input may be the concatenation [x1, upsample2(x2)] of a
// full-resolution tensor and a half-resolution one; the upsampling is done
// while loading, so the decoder never materialises the concatenation.
#include <cuda_bf16.h>

#include <cstdint>

#include "lbib_internal.cuh"
#include "nn.cuh"

namespace lbib {
namespace nn {

// eight BF16 channels (16 bytes) in and out of FP32 registers
__device__ __forceinline__ void load8(const __nv_bfloat16* p, float v[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        v[2 * k] = f.x;
        v[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void store8(__nv_bfloat16* p, const float v[8]) {
    uint4 u;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    *reinterpret_cast<uint4*>(p) = u;
}

constexpr int TH = kTH, TW = kTW, BM = TH * TW, BN = 64, KC = 32;
constexpr int HH = TH + 2, HWD = TW + 2;   // halo tile
constexpr int AST = KC + 8;                // smem row stride (bf16) of halo / weight rows
constexpr int kConvThreads = 256;
constexpr int kHaloBytes = HH * HWD * AST * 2;
constexpr int kWBytes = 9 * BN * AST * 2;
static_assert(kConvSmem == kHaloBytes + kWBytes, "conv smem");

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::);
}
__device__ __forceinline__ void ldmatrix_x4(unsigned r[4], const void* p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void ldmatrix_x4_trans(unsigned r[4], const void* p) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage the 10 x 18 halo of the pixel tile (y0, x0) for input channels
// [ci0, ci0 + KC) into `halo` (rows of AST bf16); zeros outside the image
// and beyond Ci.
__device__ __forceinline__ void load_halo(const ConvArgs& a, int n, int y0, int x0, int ci0,
                                          __nv_bfloat16* halo) {
    const int Ci = a.C1 + a.C2;
    for (int idx = threadIdx.x; idx < HH * HWD * (KC / 8); idx += blockDim.x) {
        const int hp = idx / (KC / 8), cc = idx % (KC / 8);
        const int gy = y0 + hp / HWD - 1, gx = x0 + hp % HWD - 1;
        const int ci = ci0 + cc * 8;
        const bool ok = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W && ci < Ci;
        const __nv_bfloat16* src = a.in1;
        if (ok) {
            if (ci < a.C1)
                src = a.in1 + (((int64_t)n * a.H + gy) * a.W + gx) * a.C1 + ci;
            else
                src = a.in2 + (((int64_t)n * (a.H >> 1) + (gy >> 1)) * (a.W >> 1) + (gx >> 1)) *
                                  a.C2 + (ci - a.C1);
        }
        cp_async16(halo + hp * AST + cc * 8, src, ok);
    }
}

__global__ void __launch_bounds__(kConvThreads) conv3x3_fwd_kernel(ConvArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* wts = reinterpret_cast<__nv_bfloat16*>(smem + kHaloBytes);
    const int tiles_x = (a.W + TW - 1) / TW;
    const int y0 = (blockIdx.x / tiles_x) * TH, x0 = (blockIdx.x % tiles_x) * TW;
    const int co0 = blockIdx.y * BN, n = blockIdx.z;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int Ci = a.C1 + a.C2;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    for (int ci0 = 0; ci0 < Ci; ci0 += KC) {
        load_halo(a, n, y0, x0, ci0, halo);
        for (int idx = tid; idx < 9 * BN * (KC / 8); idx += blockDim.x) {
            const int tap = idx / (BN * (KC / 8)), r = idx % (BN * (KC / 8));
            const int co = r / (KC / 8), cc = r % (KC / 8);
            const int gco = co0 + co, ci = ci0 + cc * 8;
            const bool ok = gco < a.Co && ci < Ci;
            const __nv_bfloat16* src = ok ? a.w + ((int64_t)tap * a.Co + gco) * Ci + ci : a.w;
            cp_async16(wts + (tap * BN + co) * AST + cc * 8, src, ok);
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
                unsigned af[2][4], bf[4][2];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int p = wm * 32 + mt * 16 + (lane & 15);
                    const int hrow = (p / TW + ky) * HWD + (p % TW + kx);
                    ldmatrix_x4(af[mt], halo + hrow * AST + kk * 16 + (lane >> 4) * 8);
                }
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    const int co = wn * 32 + np * 16 + (lane & 7) + 8 * (lane >> 4);
                    unsigned r[4];
                    ldmatrix_x4(r, wts + (tap * BN + co) * AST + kk * 16 + ((lane >> 3) & 1) * 8);
                    bf[np * 2][0] = r[0];
                    bf[np * 2][1] = r[1];
                    bf[np * 2 + 1][0] = r[2];
                    bf[np * 2 + 1][1] = r[3];
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
            }
        }
        __syncthreads();
    }

    // epilogue: bias, ReLU, store (pairs of output channels)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int p = wm * 32 + mt * 16 + (lane >> 2) + 8 * h;
            const int gy = y0 + p / TW, gx = x0 + p % TW;
            if (gy >= a.H || gx >= a.W) continue;
            const int64_t pix = ((int64_t)n * a.H + gy) * a.W + gx;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int co = co0 + wn * 32 + nt * 8 + (lane & 3) * 2;
                if (co >= a.Co) continue;
                float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[co];
                    if (co + 1 < a.Co) v1 += a.bias[co + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (a.gate) {
                    const __nv_bfloat16* gt = a.gate + pix * a.Co + co;
                    if (!(__bfloat162float(gt[0]) > 0.f)) v0 = 0.f;
                    if (co + 1 < a.Co && !(__bfloat162float(gt[1]) > 0.f)) v1 = 0.f;
                }
                if (a.out_f32) {
                    float* o = static_cast<float*>(a.out) + pix * a.Co + co;
                    o[0] = v0;
                    if (co + 1 < a.Co) o[1] = v1;
                } else {
                    __nv_bfloat162 pr = __floats2bfloat162_rn(v0, v1);
                    *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(a.out) +
                                                       pix * a.Co + co) = pr;
                }
            }
        }
}

// ---------------------------------------------------------------------------
// Weight gradient: dw[tap][i][o] += sum_p in(p + tap)[i] * g[p][o].  A CTA
// takes 16 input channels x 64 output channels x all 9 taps over a run of
// pixel tiles; per tile it stages the input halo and the gradient tile and
// accumulates with mma.sync (M = input channel, N = output channel, K =
// pixels, both operands read transposed by ldmatrix.trans).  The CTA's sums
// are added to the FP32 gradient with atomics.
constexpr int WCI = 16;  // input channels per CTA
constexpr int GST = BN + 8;
static_assert(kWgSmem == kHaloBytes + BM * GST * 2, "wgrad smem");

__global__ void __launch_bounds__(kConvThreads) conv3x3_wgrad_kernel(WgradArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem);
    __nv_bfloat16* gt = reinterpret_cast<__nv_bfloat16*>(smem + kHaloBytes);
    const int Ci = a.C1 + a.C2;
    const int tiles_x = (a.W + TW - 1) / TW, tiles_y = (a.H + TH - 1) / TH;
    const int tiles = tiles_x * tiles_y * a.N;
    const int ci0 = blockIdx.y * WCI, co0 = blockIdx.z * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;  // warp = n8 tile
    ConvArgs ca;
    ca.in1 = a.in1;
    ca.in2 = a.in2;
    ca.H = a.H;
    ca.W = a.W;
    ca.C1 = a.C1;
    ca.C2 = a.C2;
    float acc[9][4];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[t][k] = 0.f;
    float dbs = 0.f;

    const int t_begin = blockIdx.x * a.tiles_per_cta;
    const int t_end = min(tiles, t_begin + a.tiles_per_cta);
    for (int tile = t_begin; tile < t_end; ++tile) {
        const int n = tile / (tiles_x * tiles_y), r = tile % (tiles_x * tiles_y);
        const int y0 = (r / tiles_x) * TH, x0 = (r % tiles_x) * TW;
        // the halo holds channels [ci0 - ci0 % KC, +KC): only WCI of them are used
        const int cbase = ci0 - (ci0 % KC);
        load_halo(ca, n, y0, x0, cbase, halo);
        for (int idx = tid; idx < BM * (BN / 8); idx += blockDim.x) {
            const int p = idx / (BN / 8), cc = idx % (BN / 8);
            const int gy = y0 + p / TW, gx = x0 + p % TW, co = co0 + cc * 8;
            const bool ok = gy < a.H && gx < a.W && co < a.Co;
            const __nv_bfloat16* src =
                ok ? a.g + (((int64_t)n * a.H + gy) * a.W + gx) * a.Co + co : a.g;
            cp_async16(gt + p * GST + cc * 8, src, ok);
        }
        cp_async_wait_all();
        __syncthreads();
        const int coff = ci0 - cbase;  // 0 or 16 within the staged chunk
        if (a.db && tid < BN) {
            for (int p = 0; p < BM; ++p) dbs += __bfloat162float(gt[p * GST + tid]);
        }
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
#pragma unroll
            for (int kk = 0; kk < BM / 16; ++kk) {
                // A = in^T (16 channels x 16 pixels): rows of the halo are pixels
                unsigned af[4];
                {
                    // matrices: (ch 0-7, px 0-7), (ch 8-15, px 0-7), (ch 0-7, px 8-15),
                    // (ch 8-15, px 8-15); transposed loads of [pixel][channel] rows
                    const int m = lane >> 3;
                    const int p = kk * 16 + (lane & 7) + 8 * (m >> 1);
                    const int ch = coff + 8 * (m & 1);
                    const int hrow = (p / TW + ky) * HWD + (p % TW + kx);
                    ldmatrix_x4_trans(af, halo + hrow * AST + ch);
                }
                // B = g (16 pixels x 8 output channels of this warp)
                unsigned b[4];
                {
                    const int m = lane >> 3;
                    const int p = kk * 16 + (lane & 7) + 8 * (m & 1);
                    ldmatrix_x4_trans(b, gt + p * GST + warp * 8);
                }
                mma_bf16(acc[tap], af, b[0], b[1]);
            }
        }
        __syncthreads();
    }
    // accumulate: acc[tap] is the 16 x 8 block (channel row, output col)
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = ci0 + (lane >> 2) + 8 * h;
            const int o = co0 + warp * 8 + (lane & 3) * 2;
            if (i < Ci) {
                float* d = a.dw + ((int64_t)tap * Ci + i) * a.Co + o;
                if (o < a.Co) atomicAdd(d, acc[tap][2 * h]);
                if (o + 1 < a.Co) atomicAdd(d + 1, acc[tap][2 * h + 1]);
            }
        }
    if (a.db && tid < BN && co0 + tid < a.Co && blockIdx.y == 0) atomicAdd(a.db + co0 + tid, dbs);
}

// ---------------------------------------------------------------------------
// elementwise layers
__global__ void avgpool2_kernel(const __nv_bfloat16* x, __nv_bfloat16* y, int N, int H, int W,
                                int C) {
    // one thread: eight channels of one output pixel (C a multiple of 8)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2, C8 = C / 8;
    if (i >= (int64_t)N * Ho * Wo * C8) return;
    const int c = (int)(i % C8) * 8;
    const int64_t p = i / C8;
    const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), n = (int)(p / ((int64_t)Wo * Ho));
    const int64_t b = (((int64_t)n * H + 2 * yo) * W + 2 * xo) * C + c;
    float a[8], bb[8], cc[8], d[8], o[8];
    load8(x + b, a);
    load8(x + b + C, bb);
    load8(x + b + (int64_t)W * C, cc);
    load8(x + b + (int64_t)W * C + C, d);
#pragma unroll
    for (int k = 0; k < 8; ++k) o[k] = 0.25f * (a[k] + bb[k] + cc[k] + d[k]);
    store8(y + p * C + c, o);
}

// gx (full res) = 0.25 * g (half res) at each of the 4 children
__global__ void avgpool2_bwd_kernel(const __nv_bfloat16* g, __nv_bfloat16* gx, int N, int H,
                                    int W, int C) {
    // one thread: eight channels of one full-resolution pixel
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int C8 = C / 8;
    if (i >= (int64_t)N * H * W * C8) return;
    const int c = (int)(i % C8) * 8;
    const int64_t p = i / C8;
    const int x = (int)(p % W), y = (int)((p / W) % H), n = (int)(p / ((int64_t)W * H));
    float v[8];
    load8(g + (((int64_t)n * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] *= 0.25f;
    store8(gx + p * C + c, v);
}

// split the gradient of a concatenation [skip (C1), upsample2(x2) (C2)]:
// gskip += g[..., :C1]; gx2 (half res) = sum over the 2x2 children of g[..., C1:],
// zero where !(gate2 > 0) when gate2 (x2's ReLU output) is given
__global__ void concat_bwd_kernel(const __nv_bfloat16* g, __nv_bfloat16* gskip,
                                  __nv_bfloat16* gx2, const __nv_bfloat16* gate2, int N, int H,
                                  int W, int C1, int C2, int accumulate_skip) {
    // one thread: eight channels (C1 and C2 multiples of 8)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int C = C1 + C2, C18 = C1 / 8, C28 = C2 / 8;
    const int64_t nfull = (int64_t)N * H * W * C18;
    if (i < nfull) {
        const int c = (int)(i % C18) * 8;
        const int64_t p = i / C18;
        float v[8];
        load8(g + p * C + c, v);
        if (accumulate_skip) {
            float s0[8];
            load8(gskip + p * C1 + c, s0);
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = s0[k] + v[k];
        }
        store8(gskip + p * C1 + c, v);
        return;
    }
    const int64_t j = i - nfull;
    const int Ho = H / 2, Wo = W / 2;
    if (j >= (int64_t)N * Ho * Wo * C28) return;
    const int c = (int)(j % C28) * 8;
    const int64_t p = j / C28;
    const int xo = (int)(p % Wo), yo = (int)((p / Wo) % Ho), n = (int)(p / ((int64_t)Wo * Ho));
    float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            float v[8];
            load8(g + (((int64_t)n * H + 2 * yo + dy) * W + 2 * xo + dx) * C + C1 + c, v);
#pragma unroll
            for (int k = 0; k < 8; ++k) s8[k] += v[k];
        }
    if (gate2) {
        float gt[8];
        load8(gate2 + p * C2 + c, gt);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (!(gt[k] > 0.f)) s8[k] = 0.f;
    }
    store8(gx2 + p * C2 + c, s8);
}

// g (bf16) = g + h where act > 0, else 0 (the sum's ReLU backward)
__global__ void add_gate_kernel(__nv_bfloat16* g, const __nv_bfloat16* h,
                                const __nv_bfloat16* act, int64_t n) {
    // one thread: eight elements (n a multiple of 8)
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 8;
    if (i >= n) return;
    float a[8], b[8], t[8];
    load8(g + i, a);
    load8(h + i, b);
    load8(act + i, t);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = t[k] > 0.f ? a[k] + b[k] : 0.f;
    store8(g + i, a);
}

// MSE: loss += sum (y - t)^2 / n; dy = 2 (y - t) / n  (y in channel 0 of Cy)
__global__ void mse_kernel(const float* y, int Cy, const float* t, __nv_bfloat16* dy, int Cdy,
                           int64_t n, double* loss) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (i < n) {
        const float d = y[i * Cy] - t[i];
        d2 = d * d;
        for (int c = 0; c < Cdy; ++c)
            dy[i * Cdy + c] = __float2bfloat16(c == 0 ? 2.f * d / (float)n : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, (double)d2 / (double)n);
}

// Adam on FP32 master weights (bias-corrected, step t >= 1)
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of one layer's FP32 weights (3,3,Ci,Co):
//   wf[tap][o][i] = w[tap][i][o]          (forward: output channel rows)
//   wd[tap][i][o] = w[8 - tap][i][o]      (data gradient: flipped taps)
// padded to Cip >= Ci input and Cop >= Co output channels with zeros
__global__ void weight_copies_kernel(const float* w, int Ci, int Co, int Cip, int Cop,
                                     __nv_bfloat16* wf, __nv_bfloat16* wd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 9LL * Cip * Cop) return;
    const int o = (int)(idx % Cop);
    const int i = (int)((idx / Cop) % Cip);
    const int tap = (int)(idx / ((int64_t)Cop * Cip));
    const float v = (i < Ci && o < Co) ? w[((int64_t)tap * Ci + i) * Co + o] : 0.f;
    wf[((int64_t)tap * Cop + o) * Cip + i] = __float2bfloat16(v);
    wd[((int64_t)(8 - tap) * Cip + i) * Cop + o] = __float2bfloat16(v);
}

// network input: [mask, source, (D - 0.125)/0.075, log10(decay) + 3, 0 x 12]
__global__ void features_kernel(const uint8_t* id_mask, const uint8_t* src, const float* Dn,
                                const float* Kn, __nv_bfloat16* x, int N, int HW) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * HW) return;
    const int n = (int)(i / HW);
    float v[8] = {id_mask[i] ? 1.f : 0.f, src[i] ? 1.f : 0.f, Dn[n], Kn[n], 0.f, 0.f, 0.f, 0.f};
    const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    store8(x + i * 16, v);
    store8(x + i * 16 + 8, z);
}

// target y = phi * decay / src_rate; prediction phi = y * src_rate / decay
__global__ void scale_kernel(const float* in, int Cin, float* out, const float* fac, int N,
                             int HW) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * HW) return;
    out[i] = in[i * Cin] * fac[i / HW];
}

}  // namespace nn
}  // namespace lbib
