// conv_tc.cu -- the 3x3 convolutions of the neural operator on the fifth-
// generation tensor cores: tcgen05.mma (BF16 operands, FP32 accumulation)
// with the accumulators in tensor memory (TMEM), operands staged in shared
// memory by the tensor memory accelerator (TMA), one thread issuing copies
// and matrix multiplies, mbarriers pacing up to three pipeline stages.
//
// Implicit GEMM: M = output pixels, N = the output channels (rounded up to
// 16, split into equal tiles of at most 128 -- 192 for 16-channel chunks --
// one per CTA column of the grid), K = 9 taps x input channels, in chunks of
// Kc = 32 channels (16 where the channel count is not a multiple of 32).
//
// A CTA takes TR image rows of a tile of Wt columns (Wt = W up to 128, else
// 128) and stages their halo once per chunk: (TR + 2) rows of rs = Wt + 2
// pixels, one pixel per 2 Kc-byte row of shared memory, swizzled in the 32-
// or 64-byte pattern of the matching TMA mode -- one 4-D box (Kc channels x
// rs x (TR + 2) x 1 image), whose out-of-bounds fill is the image's zero
// padding.  In that layout the pixel at halo position p + ky rs + kx is tap
// (ky, kx) of output position p, so every tap of an accumulator's 128 output
// positions is one K-major operand starting ky rs + kx rows further on: the
// tensor cores read swizzled operands from any row (the swizzle follows the
// absolute shared-memory address, and the stages are 1024-byte aligned).
// Accumulators of 128 TMEM lanes:
//   Wt = 128: one per image row (m = TR), lane = column;
//   Wt < 128: m = ceil(TR rs / 128) over the row-major halo positions, the
//   two lanes per row that fall on halo columns discarded.
// The decoder's upsampled half-resolution channels (each value repeated 2 x
// 2) are staged by the threads with cp.async into the same swizzled layout.
// The weights are pre-tiled and pre-swizzled (tile_weights_tc_kernel) into
// [N tile][chunk][tap][output channel][Kc input channels], so that one bulk
// copy loads a chunk's weights for all nine taps.
//
// Every mbarrier wait is bounded: a wait that runs out raises the error word,
// the CTA waits (again bounded) for its copies and multiplies in flight,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>

#include "lbib_internal.cuh"
#include "nn.cuh"

namespace lbib {
namespace nn {

constexpr int kTcThreads = 128;  // four warps: the accumulators' four lane quarters
constexpr int kTcM = 128;
constexpr int kTcMaxStages = 3;

struct ConvTcArgs {
    const __nv_bfloat16* in2;  // (N, H/2, W/2, C2), read upsampled, or NULL
    const __nv_bfloat16* wt;   // tiled weights, [N tiles][nk][9][Np][Kc] swizzled
    const float* bias;         // (Co) or NULL
    void* out;                 // (N, H, W, Co) bf16, or fp32 when out_f32
    const __nv_bfloat16* gate; // (N, H, W, Co) or NULL: out = 0 where !(gate > 0)
    unsigned* err;             // raised when a bounded wait runs out
    int N, H, W, C1, C2, Co;
    int Kc;                    // input channels of a chunk (32 or 16)
    int swb;                   // bytes of one staged pixel: 2 Kc, the swizzle span
    int swcode;                // the descriptors' layout code of that swizzle
    int nk, nk1;               // chunks in all, and from in1
    int Np;                    // output channels of one CTA (N tile)
    int Wt, rs, TR, m, wide;   // tile: TR rows x Wt columns, halo rows of rs pixels
    int tiles_x, tiles_y;
    int a_bytes;               // the halo region of a stage (1024-byte multiple)
    int box_bytes;             // bytes one TMA box delivers: (TR + 2) rs swb
    int stage_bytes, stages;   // stage: halo + the chunk's weights (+ the upsampled box)
    int tmem_cols;             // power of two >= max(32, m Np)
    int up_rows, up_cols;      // the half-resolution box of an upsampled chunk
    int up_off, up_box_bytes;  // its place in the stage, the bytes it delivers
    int relu, out_f32;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarriers
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_tx_only(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// a bounded wait (about a second at most): false when it ran out
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    for (int i = 0; i < (1 << 24); ++i) {
        if (mbar_try_wait(a, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

// ---- bulk copies (TMA)
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// ---- tensor memory and the tensor cores
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared memory matrix descriptor of a K-major operand in a swizzled layout:
// start address (16-byte units, bits 0-13), the leading byte offset (unused
// when one MMA's 16 K elements lie within a swizzled row; 1 by convention,
// bits 16-29), the byte distance between groups of 8 rows (bits 32-45), the
// descriptor version of this architecture (bits 46-47 = 1), base offset 0
// (bits 49-51), and the layout code (bits 61-63: 6 = 32-byte, 4 = 64-byte,
// 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t addr, uint32_t sbo, uint32_t code) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)code << 61);
}
// The same for an MN-major operand: the leading byte offset is the distance
// between M (or N) atoms, the stride byte offset between groups of 8 K rows.
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                                 uint32_t code) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)code << 61);
}
// Byte offset, within a 1024-byte aligned region, of the 16-byte piece that
// the TMA's swizzle of span swb places at the unswizzled offset off: bits 4..
// of the piece index XOR the bits from 7 on (one bit for 32 bytes, two for 64,
// three for 128).
__host__ __device__ __forceinline__ uint32_t swizzle_off(uint32_t off, int swb) {
    return off ^ (((off >> 7) & (uint32_t)((swb >> 4) - 1)) << 4);
}

// The decoder's upsampled channels: the half-resolution box (staged by TMA in
// the same swizzle, origin at half-resolution pixel ((x0 - 1) >> 1,
// (y0 - 1) >> 1), up_cols wide) expanded into the halo layout -- halo pixel hp
// (row hp / rs, column hp % rs of the halo starting at (x0 - 1, y0 - 1))
// takes half-resolution pixel (gy >> 1, gx >> 1).  Outside the image the box
// holds the TMA's zero fill, which is the zero padding (H and W are even).
__device__ __forceinline__ void expand_upsampled(unsigned char* dst, const unsigned char* stg,
                                                 int halo_rows, int rs, int swb, int x0, int y0,
                                                 int up_cols, int tid, int nthreads) {
    const int ppp = swb / 16;
    const int by = (y0 - 1) >> 1, bx = (x0 - 1) >> 1;
    for (int i = tid; i < halo_rows * rs * ppp; i += nthreads) {
        const int hp = i / ppp, q = i % ppp;
        const int gy = y0 - 1 + hp / rs, gx = x0 - 1 + hp % rs;
        const int srow = ((gy >> 1) - by) * up_cols + ((gx >> 1) - bx);
        const uint4 v = *reinterpret_cast<const uint4*>(
            stg + swizzle_off((uint32_t)(srow * swb + q * 16), swb));
        *reinterpret_cast<uint4*>(dst + swizzle_off((uint32_t)(hp * swb + q * 16), swb)) = v;
    }
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major, N / 8 in bits 17-22,
// M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                     "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}


// UP: the layer has upsampled channels (the expansion is compiled only then)
template <bool UP>
__global__ void __launch_bounds__(kTcThreads)
    conv3x3_tc_kernel(const __grid_constant__ CUtensorMap map1,
                      const __grid_constant__ CUtensorMap map2, ConvTcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kTcMaxStages], bar_done[kTcMaxStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_bad, s_committed, s_up_ok;
    // stages at 1024-byte boundaries: the swizzle follows the address bits
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = a.stages;

    const int per_img = a.tiles_x * a.tiles_y;
    const int n = blockIdx.x / per_img;
    const int rem = blockIdx.x % per_img;
    const int y0 = (rem / a.tiles_x) * a.TR, x0 = (rem % a.tiles_x) * a.Wt;
    const int co0 = blockIdx.y * a.Np;  // this CTA's output channels
    const __nv_bfloat16* wt = a.wt + (int64_t)blockIdx.y * a.nk * 9 * a.Np * a.Kc;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_done[s]), 1);
        }
        s_bad = 0;
        s_committed = -1;  // the last chunk whose multiplies were committed
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = mma_idesc(kTcM, a.Np);
    const uint32_t b_bytes = 9u * (uint32_t)a.Np * (uint32_t)a.swb;
    const uint32_t sbo = 8u * (uint32_t)a.swb;
    // thread 0: per stage, the chunk whose copies were issued and not yet
    // waited for (-1 = none)
    int loading[kTcMaxStages] = {-1, -1, -1};

    auto issue = [&](int k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        const uint32_t fb = smem_u32(&bar_full[s]);
        if (!UP || k < a.nk1) {
            mbar_expect_tx(fb, b_bytes + (uint32_t)a.box_bytes);
            tma_load_4d(st, &map1, k * a.Kc, x0 - 1, y0 - 1, n, fb);
        } else {
            mbar_expect_tx(fb, b_bytes + (uint32_t)a.up_box_bytes);
            tma_load_4d(st + (uint32_t)a.up_off, &map2, (k - a.nk1) * a.Kc, (x0 - 1) >> 1,
                        (y0 - 1) >> 1, n, fb);
        }
        bulk_load(st + (uint32_t)a.a_bytes, wt + (int64_t)k * 9 * a.Np * a.Kc, b_bytes, fb);
        loading[s] = k;
    };

    // an upsampled chunk: once its half-resolution box has landed the threads
    // expand it into the halo (the stage's previous multiplies completed
    // before its copies were issued); done one chunk ahead, beside the
    // multiplies of the chunk before
    auto expand_chunk = [&](int k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        if (tid == 0) {
            s_up_ok = !s_bad && mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1) ? 1 : 0;
            if (!s_up_ok) s_bad = 1;
        }
        __syncthreads();
        if (s_up_ok && mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
            unsigned char* gst = smem_raw + (st - smem_u32(smem_raw));
            expand_upsampled(gst, gst + a.up_off, a.TR + 2, a.rs, a.swb, x0, y0, a.up_cols, tid,
                             kTcThreads);
        }
        // written through the generic proxy, read by the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    if (tid == 0)
        for (int k = 0; k < NS && k < a.nk; ++k) issue(k);
    if (UP && a.nk1 == 0) {
        expand_chunk(0);
        __syncthreads();
    }
    for (int k = 0; k < a.nk; ++k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
                s_bad = 1;
            } else {
                loading[s] = -1;
                tc_fence_after();
                const uint32_t bst = st + (uint32_t)a.a_bytes;
                for (int t = 0; t < 9; ++t) {
                    const int ky = t / 3, kx = t % 3;
                    for (int kk = 0; kk < a.Kc / 16; ++kk) {
                        const uint64_t bdesc = smem_desc_sw(
                            bst + (uint32_t)(t * a.Np * a.swb + kk * 32), sbo, (uint32_t)a.swcode);
                        for (int j = 0; j < a.m; ++j) {
                            const int row = (a.wide ? j * a.rs : j * kTcM) + ky * a.rs + kx;
                            const uint64_t adesc = smem_desc_sw(
                                st + (uint32_t)(row * a.swb + kk * 32), sbo, (uint32_t)a.swcode);
                            tc_mma(tmem + (uint32_t)(j * a.Np), adesc, bdesc, idesc,
                                   (k > 0 || t > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                }
                tc_commit(smem_u32(&bar_done[s]));
                s_committed = k;
                // refill the stage of chunk k - 1, whose multiplies ran ahead
                // of the ones just issued
                if (k >= 1 && k - 1 + NS < a.nk) {
                    if (!mbar_wait(smem_u32(&bar_done[(k - 1) % NS]), ((k - 1) / NS) & 1))
                        s_bad = 1;
                    else
                        issue(k - 1 + NS);
                }
            }
        }
        if (UP && k + 1 < a.nk && k + 1 >= a.nk1) expand_chunk(k + 1);
        __syncthreads();
        if (s_bad) break;
    }
    // after an error: the copies still in flight land before the CTA leaves
    if (tid == 0)
        for (int s = 0; s < NS; ++s)
            if (loading[s] >= 0) mbar_wait(smem_u32(&bar_full[s]), (loading[s] / NS) & 1);
    __syncthreads();
    // the last commit covers every multiply issued before it
    const int committed = s_committed;
    bool ok = !s_bad;
    if (committed >= 0 && !mbar_wait(smem_u32(&bar_done[committed % NS]), (committed / NS) & 1))
        ok = false;
    tc_fence_after();

    if (ok) {
        // epilogue: warp w owns lanes 32w .. 32w + 31 of every accumulator
        const int i = warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j = 0; j < a.m; ++j) {
            const int lin = j * kTcM + i;
            const int r = a.wide ? j : lin / a.rs, c = a.wide ? i : lin % a.rs;
            const bool valid = c < a.Wt && r < a.TR && y0 + r < a.H;
            const int64_t pix = ((int64_t)n * a.H + y0 + r) * a.W + x0 + c;
            for (int cl = 0; cl < a.Np; cl += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)(j * a.Np + cl), v);
                if (!valid) continue;
                const int c0 = co0 + cl;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int co = c0 + q;
                    if (co < a.Co) {
                        if (a.bias) v[q] += a.bias[co];
                        if (a.relu) v[q] = fmaxf(v[q], 0.f);
                    }
                }
                if (a.gate) {
                    const __nv_bfloat16* gt = a.gate + pix * a.Co + c0;
                    if (c0 + 16 <= a.Co && (a.Co % 8) == 0) {
                        __nv_bfloat162 h[8];
                        const uint4 g0 = __ldg(reinterpret_cast<const uint4*>(gt));
                        const uint4 g1 = __ldg(reinterpret_cast<const uint4*>(gt) + 1);
                        std::memcpy(&h[0], &g0, 16);
                        std::memcpy(&h[4], &g1, 16);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float2 f = __bfloat1622float2(h[q]);
                            if (!(f.x > 0.f)) v[2 * q] = 0.f;
                            if (!(f.y > 0.f)) v[2 * q + 1] = 0.f;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (c0 + q < a.Co && !(__bfloat162float(gt[q]) > 0.f)) v[q] = 0.f;
                    }
                }
                if (a.out_f32) {
                    float* o = static_cast<float*>(a.out) + pix * a.Co;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (c0 + q < a.Co) o[c0 + q] = v[q];
                } else {
                    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.out) + pix * a.Co + c0;
                    if (c0 + 16 <= a.Co && (a.Co % 8) == 0) {
                        uint4 w0, w1;
                        __nv_bfloat162 h[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        std::memcpy(&w0, &h[0], 16);
                        std::memcpy(&w1, &h[4], 16);
                        reinterpret_cast<uint4*>(o)[0] = w0;
                        reinterpret_cast<uint4*>(o)[1] = w1;
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (c0 + q < a.Co) o[q] = __float2bfloat16_rn(v[q]);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(a.err, 1u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tmem_cols)
                     : "memory");
}

// Weights (9, Co, Ci) -> [N tiles][Ci / Kc chunks][9 taps][Np output
// channels][Kc input channels], each output channel's row of 2 Kc bytes
// swizzled as the TMA would place it in a 1024-byte aligned region (a tap's
// block of Np rows is a multiple of the swizzle's repeat); zeros for output
// channels >= Co.
__global__ void tile_weights_tc_kernel(const __nv_bfloat16* w, int Co, int Ci, int Kc, int Np,
                                       int nk, int ntiles, __nv_bfloat16* wt) {
    const int64_t per_tile = (int64_t)nk * 9 * Np * Kc;
    const int64_t total = per_tile * ntiles;
    const int swb = 2 * Kc;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % per_tile;
        const int tile = (int)(i / per_tile);
        const int e = (int)(r % Kc);  // element of the unswizzled row
        const int row = (int)((r / Kc) % Np);
        const int t = (int)((r / ((int64_t)Kc * Np)) % 9);
        const int k = (int)(r / ((int64_t)Kc * Np * 9));
        const int co = tile * Np + row;
        const int ci = k * Kc + e;
        const uint32_t off = swizzle_off((uint32_t)(row * swb + e * 2), swb);
        const int64_t dst = i - e - (int64_t)row * Kc + off / 2;
        wt[dst] = (co < Co && ci < Ci) ? w[((int64_t)t * Co + co) * Ci + ci] : __float2bfloat16(0.f);
    }
}

// ---------------------------------------------------------------------------
// The weight gradient on the tensor cores: dW[ky][kx][ci][co] = sum over
// pixels p of X[p + (ky - 1, kx - 1)][ci] G[p][co], a GEMM with the pixels as
// K.  Both operands are staged as pixel rows (channels contiguous), so they
// enter the MMA MN-major: A rows (M) are input channels, B rows (N) output
// channels, K runs down the pixel rows.  The X halo of a tile (TR + 2 rows of
// rs = Wt + 2 pixels, one Kc-channel chunk, swizzled as in the forward
// kernel) makes every tap a row-shifted window, and the MN-major A operand
// puts four such windows side by side: its M atoms (Kc channels each) sit one
// pixel row apart (LBO = one row), so M = 128 covers the taps kx = 0, 1, 2
// (and a fourth, unused shift) of one ky for 32 channels -- with 16-channel
// chunks eight shifts, three of them used.  The K steps walk the tile's image
// rows 16 pixels at a time (Wt a multiple of 16), so the halo columns never
// enter: G is staged without halo, 16 output channels per TMA box (32-byte
// swizzle), its N atoms a region apart.  One accumulator per ky and per
// "set" of image rows (rows r % sets; more independent accumulation chains
// in flight), summed at the end and added to dW with FP32 reductions.  A CTA
// takes one input-channel chunk, one N tile and a range of pixel tiles
// (split K over CTAs).  Pipeline and bounded waits as the forward kernel.
constexpr int kTcMaxChunks = 24;  // input-channel chunks of a weight gradient (up to 384 channels)

struct WgTcArgs {
    const __nv_bfloat16* in2;  // (N, H/2, W/2, C2), read upsampled, or NULL
    float* dw;                 // (9, Ci, Co) FP32, accumulated
    float* db;                 // (Co) FP32, accumulated, or NULL
    unsigned* err;
    int N, H, W, C1, C2, Co;
    // the input-channel chunks (one per CTA row of the grid): 32 channels where
    // the input allows, 16 for a remainder; each from in1 or the upsampled in2
    int nchunks;
    int ck_c0[kTcMaxChunks];    // first channel within its own input
    int ck_row[kTcMaxChunks];   // first channel of dW (in1 channels, then in2's)
    int ck_kc[kTcMaxChunks];    // 32 or 16
    int ck_up[kTcMaxChunks];    // from in2
    int Np, ng;                // output channels of the N tile, its 16-channel G atoms
    int Wt, rs, TR, tiles_x, tiles_y, total_tiles;
    int sk;                    // CTAs sharing one (chunk, N tile): split K
    int sets;                  // accumulator sets
    int x_bytes, x_box_bytes;  // the X halo region of a stage, one TMA box
    int g_atom_bytes;          // one G atom region (TR Wt 32 bytes)
    int stage_bytes, stages, tmem_cols;
    int up_rows, up_cols, up_off, up_box_bytes;  // the half-resolution box, as in ConvTcArgs
};

template <bool UP>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv3x3_wgrad_tc_kernel(const __grid_constant__ CUtensorMap mapx32,
                            const __grid_constant__ CUtensorMap mapx16,
                            const __grid_constant__ CUtensorMap mapu32,
                            const __grid_constant__ CUtensorMap mapu16,
                            const __grid_constant__ CUtensorMap mapg, WgTcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kTcMaxStages], bar_done[kTcMaxStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_bad, s_committed, s_up_ok;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = a.stages;
    const int chunk = blockIdx.y, ntile = blockIdx.z;
    const int co0 = ntile * a.Np;
    // this CTA's chunk: its width (the 64- or 32-byte swizzle, 4 or 8 shifts
    // in M), its place in its input and in dW
    const int Kc = a.ck_kc[chunk], swx = 2 * Kc, swcode = Kc == 32 ? 4 : 6;
    const int c0 = a.ck_c0[chunk], row0 = a.ck_row[chunk];
    const bool up = UP && a.ck_up[chunk] != 0;  // the chunk comes from the upsampled input
    const CUtensorMap* mapx = Kc == 32 ? &mapx32 : &mapx16;
    const CUtensorMap* mapu = Kc == 32 ? &mapu32 : &mapu16;
    const uint32_t x_box_bytes = (uint32_t)((a.TR + 2) * a.rs * swx);
    const uint32_t up_box_bytes = (uint32_t)(a.up_rows * a.up_cols * swx);
    // this CTA's pixel tiles
    const int t_begin = (int)((int64_t)a.total_tiles * blockIdx.x / a.sk);
    const int t_end = (int)((int64_t)a.total_tiles * (blockIdx.x + 1) / a.sk);
    const int nt = t_end - t_begin;
    const int per_img = a.tiles_x * a.tiles_y;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_done[s]), 1);
        }
        s_bad = 0;
        s_committed = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    // M = 128 (the Kc-channel atoms of natoms shifts), N = Np, both MN-major
    const uint32_t idesc = mma_idesc(kTcM, a.Np) | (1u << 15) | (1u << 16);
    const uint32_t g_bytes = (uint32_t)a.ng * (uint32_t)a.g_atom_bytes;
    int loading[kTcMaxStages] = {-1, -1, -1};
    uint32_t started = 0u;  // accumulators that hold a first product
    // the CTAs of the first chunk also sum the bias gradient, in warps 1 - 3
    // (warp 0 issues the multiplies): channels tid - 32 and tid + 64 of the N tile
    const bool dbsum = a.db != nullptr && chunk == 0 && tid >= 32 && tid - 32 < a.Np;
    float db_acc[2] = {0.f, 0.f};

    auto tile_xy = [&](int T, int& n, int& y0, int& x0) {
        n = T / per_img;
        const int rem = T % per_img;
        y0 = (rem / a.tiles_x) * a.TR;
        x0 = (rem % a.tiles_x) * a.Wt;
    };
    auto issue = [&](int k) {  // local tile k of this CTA
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        const uint32_t fb = smem_u32(&bar_full[s]);
        int n, y0, x0;
        tile_xy(t_begin + k, n, y0, x0);
        if (!up) {
            mbar_expect_tx(fb, g_bytes + x_box_bytes);
            tma_load_4d(st, mapx, c0, x0 - 1, y0 - 1, n, fb);
        } else {
            mbar_expect_tx(fb, g_bytes + up_box_bytes);
            tma_load_4d(st + (uint32_t)a.up_off, mapu, c0, (x0 - 1) >> 1, (y0 - 1) >> 1, n, fb);
        }
        for (int at = 0; at < a.ng; ++at)
            tma_load_4d(st + (uint32_t)a.x_bytes + (uint32_t)(at * a.g_atom_bytes), &mapg,
                        co0 + 16 * at, x0, y0, n, fb);
        loading[s] = k;
    };

    // an upsampled chunk: each tile's half-resolution box expanded into the
    // halo one tile ahead, beside the multiplies of the tile before
    auto expand_tile = [&](int k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        int n, y0, x0;
        tile_xy(t_begin + k, n, y0, x0);
        if (tid == 0) {
            s_up_ok = !s_bad && mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1) ? 1 : 0;
            if (!s_up_ok) s_bad = 1;
        }
        __syncthreads();
        if (s_up_ok && mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
            unsigned char* gst = smem_raw + (st - smem_u32(smem_raw));
            expand_upsampled(gst, gst + a.up_off, a.TR + 2, a.rs, swx, x0, y0, a.up_cols, tid,
                             kTcThreads);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    if (tid == 0)
        for (int k = 0; k < NS && k < nt; ++k) issue(k);
    if (up && nt > 0) {
        expand_tile(0);
        __syncthreads();
    }
    for (int k = 0; k < nt; ++k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
                s_bad = 1;
            } else {
                loading[s] = -1;
                tc_fence_after();
                const uint32_t gst = st + (uint32_t)a.x_bytes;
                for (int r = 0; r < a.TR; ++r) {
                    const int set = r % a.sets;
                    for (int k0 = 0; k0 < a.Wt; k0 += 16) {
                        // G: 16-channel atoms a region apart, 8 pixel rows of 32 bytes
                        const uint64_t bdesc =
                            smem_desc_mn(gst + (uint32_t)((r * a.Wt + k0) * 32),
                                         (uint32_t)a.g_atom_bytes, 256u, 6u);
                        for (int ky = 0; ky < 3; ++ky) {
                            const int acc = set * 3 + ky;
                            const uint64_t adesc = smem_desc_mn(
                                st + (uint32_t)(((r + ky) * a.rs + k0) * swx), (uint32_t)swx,
                                8u * (uint32_t)swx, (uint32_t)swcode);
                            tc_mma(tmem + (uint32_t)(acc * a.Np), adesc, bdesc, idesc,
                                   (started >> acc) & 1u);
                            started |= 1u << acc;
                        }
                    }
                }
                tc_commit(smem_u32(&bar_done[s]));
                s_committed = k;
                if (k >= 1 && k - 1 + NS < nt) {
                    if (!mbar_wait(smem_u32(&bar_done[(k - 1) % NS]), ((k - 1) / NS) & 1))
                        s_bad = 1;
                    else
                        issue(k - 1 + NS);
                }
            }
        }
        if (up && k + 1 < nt) expand_tile(k + 1);
        if (dbsum && !s_bad && mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
            // the bias gradient: this thread's output channels summed over
            // the tile's pixel rows of G in shared memory (beside the multiplies)
            for (int i = 0; i < 2; ++i) {
                const int c = tid - 32 + 96 * i;
                if (c >= a.Np) break;
                const unsigned char* g0 = smem_raw + (st - smem_u32(smem_raw)) + a.x_bytes +
                                          (c >> 4) * a.g_atom_bytes;
                const int e = c & 15;
                float acc = 0.f;
                for (int p = 0; p < a.TR * a.Wt; ++p)
                    acc += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(
                        g0 + swizzle_off((uint32_t)(p * 32 + e * 2), 32)));
                db_acc[i] += acc;
            }
        }
        __syncthreads();
        if (s_bad) break;
    }
    if (tid == 0)
        for (int s = 0; s < NS; ++s)
            if (loading[s] >= 0) mbar_wait(smem_u32(&bar_full[s]), (loading[s] / NS) & 1);
    __syncthreads();
    const int committed = s_committed;
    bool ok = !s_bad;
    if (committed >= 0 && !mbar_wait(smem_u32(&bar_done[committed % NS]), (committed / NS) & 1))
        ok = false;
    tc_fence_after();

    if (ok && committed >= 0) {
        // lane m of warp w: A row m = 32 w + lane = (shift j, channel ci)
        const int m = warp * 32 + lane;
        const int j = m / Kc, ci = m % Kc;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int ky = 0; ky < 3; ++ky)
            for (int cl = 0; cl < a.Np; cl += 16) {
                float v[16], w[16];
                __syncwarp();
                tmem_ld16(trow + (uint32_t)(ky * a.Np + cl), v);
                for (int set = 1; set < a.sets; ++set) {
                    __syncwarp();
                    tmem_ld16(trow + (uint32_t)((set * 3 + ky) * a.Np + cl), w);
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] += w[q];
                }
                if (j < 3) {
                    float* d = a.dw + ((int64_t)(ky * 3 + j) * (a.C1 + a.C2) + row0 + ci) * a.Co +
                               co0 + cl;
                    if (co0 + cl + 16 <= a.Co) {
                        // four FP32 reductions per instruction (d is 16-byte aligned:
                        // Co and co0 + cl are multiples of 16)
#pragma unroll
                        for (int q = 0; q < 16; q += 4)
                            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(d + q),
                                         "f"(v[q]), "f"(v[q + 1]), "f"(v[q + 2]), "f"(v[q + 3])
                                         : "memory");
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (co0 + cl + q < a.Co) atomicAdd(d + q, v[q]);
                    }
                }
            }
    } else if (!ok && tid == 0) {
        atomicOr(a.err, 1u);
    }
    if (ok && dbsum)
        for (int i = 0; i < 2; ++i) {
            const int c = tid - 32 + 96 * i;
            if (c < a.Np && co0 + c < a.Co) atomicAdd(a.db + co0 + c, db_acc[i]);
        }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(a.tmem_cols)
                     : "memory");
}

// The fused weight refresh: for layer blockIdx.y, from its FP32 master
// weights w (9, Ci, Co): the BF16 forward copy wf (9, Co, Ci), the
// tap-flipped copy wd (9, Ci, Co) (wd[8 - t][i][o] = w[t][i][o]) and the
// tcgen05 tilings of both (tile_weights_tc_kernel's layout, element values
// taken straight from w), in one grid-stride pass per layer.
struct TileGeom {
    int Kc, Np, nk, nt;
};
__device__ __forceinline__ TileGeom tile_geom(int Ci, int Co) {
    TileGeom g;
    g.Kc = Ci % 32 == 0 ? 32 : 16;
    const int n16 = (Co + 15) / 16;
    const int per = g.Kc == 32 ? 8 : 12;
    g.nt = (n16 + per - 1) / per;
    g.Np = (n16 + g.nt - 1) / g.nt * 16;
    g.nk = Ci / g.Kc;
    return g;
}
// element i of the tiling of a (9, Co, Ci) array, counted with the output
// channel (row) fastest or the input channel (e) fastest -- whichever is
// contiguous in the FP32 source, so that a warp's reads coalesce: where it
// goes (dst) and which (tap, co, ci) of the array it holds; false for padding
// (co >= Co)
__device__ __forceinline__ bool tiled_source(int64_t i, int Ci, int Co, const TileGeom& g,
                                             bool row_fast, int64_t* dst, int* t, int* co,
                                             int* ci) {
    const int64_t per_tile = (int64_t)g.nk * 9 * g.Np * g.Kc;
    const int64_t r = i % per_tile;
    const int tile = (int)(i / per_tile);
    const int row = row_fast ? (int)(r % g.Np) : (int)((r / g.Kc) % g.Np);
    const int e = row_fast ? (int)((r / g.Np) % g.Kc) : (int)(r % g.Kc);
    *t = (int)((r / ((int64_t)g.Np * g.Kc)) % 9);
    const int k = (int)(r / ((int64_t)g.Np * g.Kc * 9));
    *co = tile * g.Np + row;
    *ci = k * g.Kc + e;
    const int swb = 2 * g.Kc;
    const uint32_t off = swizzle_off((uint32_t)(row * swb + e * 2), swb);
    *dst = (int64_t)tile * per_tile + ((int64_t)k * 9 + *t) * g.Np * g.Kc + off / 2;
    return *co < Co && *ci < Ci;
}
__global__ void refresh_weights_kernel(const WeightSet* sets) {
    const WeightSet ws = sets[blockIdx.y];
    const int Ci = ws.Ci, Co = ws.Co;
    const int64_t n_copy = 9LL * Ci * Co;
    const TileGeom gf = tile_geom(Ci, Co), gd = tile_geom(Co, Ci);
    const int64_t n_f = ws.wft ? (int64_t)gf.nt * gf.nk * 9 * gf.Np * gf.Kc : 0;
    const int64_t n_d = ws.wdt ? (int64_t)gd.nt * gd.nk * 9 * gd.Np * gd.Kc : 0;
    const int64_t total = n_copy + n_f + n_d;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n_copy) {
            const int o = (int)(i % Co);
            const int in = (int)((i / Co) % Ci);
            const int t = (int)(i / ((int64_t)Co * Ci));
            const __nv_bfloat16 v = __float2bfloat16(ws.w[i]);
            ws.wf[((int64_t)t * Co + o) * Ci + in] = v;
            ws.wd[((int64_t)(8 - t) * Ci + in) * Co + o] = v;
        } else if (i < n_copy + n_f) {
            // the forward tiling: the (9, Co, Ci) array is wf
            int64_t dst;
            int t, co, ci;
            const bool in = tiled_source(i - n_copy, Ci, Co, gf, true, &dst, &t, &co, &ci);
            ws.wft[dst] = in ? __float2bfloat16(ws.w[((int64_t)t * Ci + ci) * Co + co])
                             : __float2bfloat16(0.f);
        } else {
            // the data-gradient tiling: the (9, Ci, Co) array is wd, whose
            // output channels are the forward input channels
            int64_t dst;
            int t, co, ci;
            const bool in = tiled_source(i - n_copy - n_f, Co, Ci, gd, false, &dst, &t, &co, &ci);
            ws.wdt[dst] = in ? __float2bfloat16(ws.w[((int64_t)(8 - t) * Ci + co) * Co + ci])
                             : __float2bfloat16(0.f);
        }
    }
}

}  // namespace nn

// ---------------------------------------------------------------------------
// host side

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// input channels of a K chunk: 32 (64-byte swizzle) where the channel count
// allows, else 16 (32-byte swizzle)
static int tc_kc(int Ci) { return Ci % 32 == 0 ? 32 : 16; }

// output channels per CTA: all of them (rounded up to 16) up to 128 (192 for
// 16-channel chunks), else equal tiles of at most that
static void tc_ntiles(int Co, int Kc, int* ntiles, int* Np) {
    const int n16 = (Co + 15) / 16;
    const int per = Kc == 32 ? 8 : 12;
    *ntiles = (n16 + per - 1) / per;
    *Np = (n16 + *ntiles - 1) / *ntiles * 16;
}

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
        cudaGetLastError();
    }
    return n;
}

constexpr int kTcSmemMax = 227 * 1024 - 1024;  // dynamic shared memory of one CTA
constexpr int kTcSmemSM = 228 * 1024;          // shared memory of an SM
constexpr int kTcMaxAcc = 4;                   // accumulators per CTA
constexpr int kTcMaxCols = 256;                // TMEM columns per CTA (two CTAs per SM)

// The tile plan: TR rows per CTA (m accumulators), chosen for the fraction of
// useful MMA lanes, of halo rows loaded once and of rows inside the image,
// as long as two waves of CTAs remain; up to three stages.
static bool tc_plan(int N, int H, int W, int Np, int ntiles, int nk, bool up,
                    nn::ConvTcArgs* a) {
    a->Wt = W <= 128 ? W : 128;
    a->rs = a->Wt + 2;
    a->wide = a->Wt == 128 ? 1 : 0;
    a->tiles_x = W / a->Wt;
    const int b_bytes = (9 * Np * a->swb + 1023) / 1024 * 1024;
    double best = -1.0;
    for (int TR = 1; TR <= H && TR <= 64; ++TR) {
        const int m = a->wide ? TR : (TR * a->rs + nn::kTcM - 1) / nn::kTcM;
        if (m > kTcMaxAcc || m * Np > kTcMaxCols) break;
        const int rows = a->wide ? (TR + 2) * a->rs : std::max((TR + 2) * a->rs, nn::kTcM * m + 2 * a->rs + 2);
        const int a_bytes = (rows * a->swb + 1023) / 1024 * 1024;
        // an upsampled chunk's half-resolution box (rows for either parity of y0)
        const int up_rows = (TR + 3) / 2 + 1, up_cols = a->Wt / 2 + 2;
        const int up_bytes = up ? (up_rows * up_cols * a->swb + 1023) / 1024 * 1024 : 0;
        const int stage = a_bytes + b_bytes + up_bytes;
        // three stages where they fit without costing the second CTA per SM
        int ns = nk == 1 ? 1 : 3;
        while (ns > 1 && ns * stage + 1024 > kTcSmemMax) --ns;
        if (ns == 3 && 2 * (3 * stage + 2048) > kTcSmemSM && 2 * (2 * stage + 2048) <= kTcSmemSM)
            ns = 2;
        if (ns * stage + 1024 > kTcSmemMax || (nk > 1 && ns < 2)) continue;
        const int ty = (H + TR - 1) / TR;
        const int64_t ctas = (int64_t)N * ty * a->tiles_x * ntiles;
        double score = (double)(TR * a->Wt) / (m * nn::kTcM) * TR / (TR + 2.0) * H / (double)(ty * TR);
        if (ctas < 2 * sm_count()) score *= (double)ctas / (2 * sm_count());
        if (score > best + 1e-9) {
            best = score;
            a->TR = TR;
            a->m = m;
            a->tiles_y = ty;
            a->a_bytes = a_bytes;
            a->box_bytes = (TR + 2) * a->rs * a->swb;
            a->stage_bytes = stage;
            a->stages = ns;
            a->up_rows = up_rows;
            a->up_cols = up_cols;
            a->up_off = a_bytes + b_bytes;
            a->up_box_bytes = up_rows * up_cols * a->swb;
        }
    }
    if (best < 0) return false;
    a->tmem_cols = 32;
    while (a->tmem_cols < a->m * Np) a->tmem_cols *= 2;
    return true;
}

int64_t tc_tiled_weight_elems(int Ci, int Co) {
    const int Kc = tc_kc(Ci);
    int nt, Np;
    tc_ntiles(Co, Kc, &nt, &Np);
    return (int64_t)nt * (Ci / Kc) * 9 * Np * Kc;
}

bool tc_conv_supported(int H, int W, int C1, int C2, int Co) {
    const int Ci = C1 + C2;
    if (H < 1 || W < 1 || (W > 128 && W % 128) || C1 < 16 || C1 % 16 || C2 < 0 || C2 % 16 ||
        Co < 1 || (C2 > 0 && (H % 2 || W % 2)) || C1 % tc_kc(Ci) || encode_fn() == nullptr)
        return false;
    nn::ConvTcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Kc = tc_kc(Ci);
    a.swb = 2 * a.Kc;
    int nt, Np;
    tc_ntiles(Co, a.Kc, &nt, &Np);
    return tc_plan(1, H, W, Np, nt, Ci / a.Kc, C2 > 0, &a);
}

cudaError_t tc_tile_weights(const void* w, int Co, int Ci, void* wt, cudaStream_t s) {
    const int Kc = tc_kc(Ci);
    int nt, Np;
    tc_ntiles(Co, Kc, &nt, &Np);
    const int nk = Ci / Kc;
    const int64_t total = (int64_t)nt * nk * 9 * Np * Kc;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    nn::tile_weights_tc_kernel<<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(w), Co, Ci,
                                                      Kc, Np, nk, nt,
                                                      static_cast<__nv_bfloat16*>(wt));
    return cudaGetLastError();
}

// ---- the weight gradient
// output channels of one N tile (at most 160: three accumulators of Np
// columns and more sets where they fit in the 512 TMEM columns)
static void tcw_ntiles(int Co, int* ntiles, int* Np) {
    const int n16 = (Co + 15) / 16;
    *ntiles = (n16 + 9) / 10;
    *Np = (n16 + *ntiles - 1) / *ntiles * 16;
}

bool tc_wgrad_supported(int H, int W, int C1, int C2, int Co) {
    if (H < 1 || W < 16 || (W <= 128 ? W % 16 : W % 128) || C1 < 16 || C1 % 16 || C2 < 0 ||
        C2 % 16 || Co < 16 || Co % 16 || (C2 > 0 && (H % 2 || W % 2)) ||
        (C1 + C2) > 16 * nn::kTcMaxChunks || encode_fn() == nullptr)
        return false;
    return true;
}

cudaError_t tc_conv3x3_wgrad(const nn::WgradArgs& w, unsigned* err, cudaStream_t s) {
    if (!tc_wgrad_supported(w.H, w.W, w.C1, w.C2, w.Co)) return cudaErrorInvalidValue;
    nn::WgTcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in2 = w.in2;
    a.dw = w.dw;
    a.db = w.db;
    a.err = err;
    a.N = w.N;
    a.H = w.H;
    a.W = w.W;
    a.C1 = w.C1;
    a.C2 = w.C2;
    a.Co = w.Co;
    // the chunks: 32 channels where the input has them, 16 for a remainder
    int nchunks = 0;
    for (int src = 0; src < 2; ++src) {
        const int C = src == 0 ? w.C1 : w.C2;
        for (int c = 0; c < C;) {
            if (nchunks == nn::kTcMaxChunks) return cudaErrorInvalidValue;
            const int kc = C - c >= 32 ? 32 : 16;
            a.ck_c0[nchunks] = c;
            a.ck_row[nchunks] = (src == 0 ? 0 : w.C1) + c;
            a.ck_kc[nchunks] = kc;
            a.ck_up[nchunks] = src;
            ++nchunks;
            c += kc;
        }
    }
    a.nchunks = nchunks;
    int ntn = 1;
    tcw_ntiles(w.Co, &ntn, &a.Np);
    a.ng = a.Np / 16;
    a.Wt = w.W <= 128 ? w.W : 128;
    a.rs = a.Wt + 2;
    a.tiles_x = w.W / a.Wt;
    // the tile: TR rows, the largest of 4, 2, 1 whose stage fits twice; the
    // halo region holds a 32-channel chunk (64-byte rows) plus the rows the
    // unused shifts of the last K step read (up to eight, for 16 channels)
    for (int TR = 4; TR >= 1; TR /= 2) {
        const int rows = (TR + 2) * a.rs + 8;
        const int xb = (rows * 64 + 1023) / 1024 * 1024;
        const int gab = TR * a.Wt * 32;
        const int up_rows = (TR + 3) / 2 + 1, up_cols = a.Wt / 2 + 2;
        const int up_off = (xb + a.ng * gab + 1023) / 1024 * 1024;
        const int up_bytes = w.C2 > 0 ? (up_rows * up_cols * 64 + 1023) / 1024 * 1024 : 0;
        const int stage = up_off + up_bytes;
        if (2 * stage + 1024 > kTcSmemMax && TR > 1) continue;
        a.TR = TR;
        a.x_bytes = xb;
        a.g_atom_bytes = gab;
        a.stage_bytes = stage;
        a.up_rows = up_rows;
        a.up_cols = up_cols;
        a.up_off = up_off;
        a.stages = 3 * stage + 1024 <= kTcSmemMax ? 3 : 2;
        break;
    }
    if (a.stages * a.stage_bytes + 1024 > kTcSmemMax) return cudaErrorInvalidValue;
    // accumulator sets: as many as TMEM holds (three accumulators of Np
    // columns each), at most 4 and at most the tile's rows, so that every set
    // receives products
    a.sets = std::max(1, std::min(std::min(4, a.TR), 512 / (3 * a.Np)));
    a.tmem_cols = 32;
    while (a.tmem_cols < 3 * a.sets * a.Np) a.tmem_cols *= 2;
    a.tiles_y = (w.H + a.TR - 1) / a.TR;
    a.total_tiles = w.N * a.tiles_y * a.tiles_x;
    // split K: one wave of CTAs over all (chunk, N tile) pairs (each CTA's
    // partial sums cost one reduction per weight), at least two tiles each
    a.sk = std::max(1, std::min(a.total_tiles / 2, sm_count() / (nchunks * ntn)));
    // tensor maps: the inputs (channels, x, y, image) with 32- and 16-channel
    // boxes (as the chunks need them), and the gradient
    cuuint32_t estr[4] = {1, 1, 1, 1};
    auto encode = [&](CUtensorMap* m, const __nv_bfloat16* p, int C, int Wd, int Hd, int bc,
                      int bw, int bh) {
        cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)Wd, (cuuint64_t)Hd, (cuuint64_t)w.N};
        cuuint64_t str[3] = {(cuuint64_t)C * 2, (cuuint64_t)Wd * C * 2,
                             (cuuint64_t)Hd * Wd * C * 2};
        cuuint32_t box[4] = {(cuuint32_t)bc, (cuuint32_t)bw, (cuuint32_t)bh, 1};
        return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(p),
                           dims, str, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           bc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                    : (bc == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_32B),
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap mg, mx32, mx16, mu32, mu16;
    std::memset(&mg, 0, sizeof(mg));
    if (!encode(&mg, w.g, w.Co, w.W, w.H, 16, a.Wt, a.TR)) return cudaErrorInvalidValue;
    bool need[2][2] = {{false, false}, {false, false}};  // [in2][16-channel]
    for (int k = 0; k < nchunks; ++k) need[a.ck_up[k]][a.ck_kc[k] == 16] = true;
    mx32 = mx16 = mu32 = mu16 = mg;  // placeholders for the boxes no chunk uses
    if (need[0][0] && !encode(&mx32, w.in1, w.C1, w.W, w.H, 32, a.rs, a.TR + 2))
        return cudaErrorInvalidValue;
    if (need[0][1] && !encode(&mx16, w.in1, w.C1, w.W, w.H, 16, a.rs, a.TR + 2))
        return cudaErrorInvalidValue;
    if (need[1][0] &&
        !encode(&mu32, w.in2, w.C2, w.W / 2, w.H / 2, 32, a.up_cols, a.up_rows))
        return cudaErrorInvalidValue;
    if (need[1][1] &&
        !encode(&mu16, w.in2, w.C2, w.W / 2, w.H / 2, 16, a.up_cols, a.up_rows))
        return cudaErrorInvalidValue;
    int smem = a.stages * a.stage_bytes + 1024;
    const int by_tmem = 512 / a.tmem_cols;
    smem = std::min(kTcSmemMax, std::max(smem, kTcSmemSM / (by_tmem + 1) - 1024 + 256));
    auto kern = w.C2 > 0 ? nn::conv3x3_wgrad_tc_kernel<true> : nn::conv3x3_wgrad_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(a.sk, nchunks, ntn), nn::kTcThreads, smem, s>>>(mx32, mx16, mu32, mu16, mg, a);
    return cudaGetLastError();
}

int64_t weight_set_elems(int Ci, int Co) {
    return 9LL * Ci * Co + tc_tiled_weight_elems(Ci, Co) + tc_tiled_weight_elems(Co, Ci);
}

cudaError_t refresh_weight_sets(const WeightSet* d_sets, int n, int64_t max_elems, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    const int bx = (int)std::min<int64_t>((max_elems + 255) / 256, 1024);
    nn::refresh_weights_kernel<<<dim3(bx, n), 256, 0, s>>>(d_sets);
    return cudaGetLastError();
}

cudaError_t tc_conv3x3(const nn::ConvArgs& c, const void* wt, unsigned* err, cudaStream_t s) {
    if (!tc_conv_supported(c.H, c.W, c.C1, c.C2, c.Co)) return cudaErrorInvalidValue;
    nn::ConvTcArgs a;
    std::memset(&a, 0, sizeof(a));
    a.in2 = c.in2;
    a.wt = static_cast<const __nv_bfloat16*>(wt);
    a.bias = c.bias;
    a.out = c.out;
    a.gate = c.gate;
    a.err = err;
    a.N = c.N;
    a.H = c.H;
    a.W = c.W;
    a.C1 = c.C1;
    a.C2 = c.C2;
    a.Co = c.Co;
    a.Kc = tc_kc(c.C1 + c.C2);
    a.swb = 2 * a.Kc;
    a.swcode = a.Kc == 32 ? 4 : 6;
    a.nk = (c.C1 + c.C2) / a.Kc;
    a.nk1 = c.C1 / a.Kc;
    int ntiles = 1;
    tc_ntiles(c.Co, a.Kc, &ntiles, &a.Np);
    if (!tc_plan(c.N, c.H, c.W, a.Np, ntiles, a.nk, c.C2 > 0, &a)) return cudaErrorInvalidValue;
    a.relu = c.relu;
    a.out_f32 = c.out_f32;
    // the full-resolution input as a 4-D tensor (channels, x, y, image); one
    // box is Kc channels x rs pixels x (TR + 2) rows of one image, swizzled
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    cuuint64_t dims[4] = {(cuuint64_t)c.C1, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
    cuuint64_t strides[3] = {(cuuint64_t)c.C1 * 2, (cuuint64_t)c.W * c.C1 * 2,
                             (cuuint64_t)c.H * c.W * c.C1 * 2};
    cuuint32_t box[4] = {(cuuint32_t)a.Kc, (cuuint32_t)a.rs, (cuuint32_t)(a.TR + 2), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                             const_cast<__nv_bfloat16*>(c.in1), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE,
                             a.Kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // the half-resolution input (channels, x, y, image); one box is Kc
    // channels x up_cols x up_rows of one image
    CUtensorMap map2 = map;
    if (c.C2 > 0) {
        cuuint64_t d2[4] = {(cuuint64_t)c.C2, (cuuint64_t)(c.W / 2), (cuuint64_t)(c.H / 2),
                            (cuuint64_t)c.N};
        cuuint64_t s2[3] = {(cuuint64_t)c.C2 * 2, (cuuint64_t)(c.W / 2) * c.C2 * 2,
                            (cuuint64_t)(c.H / 2) * (c.W / 2) * c.C2 * 2};
        cuuint32_t b2[4] = {(cuuint32_t)a.Kc, (cuuint32_t)a.up_cols, (cuuint32_t)a.up_rows, 1};
        r = encode_fn()(&map2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(c.in2),
                        d2, s2, b2, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        a.Kc == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    int smem = a.stages * a.stage_bytes + 1024;
    // no more CTAs on an SM than its tensor memory holds, so that no
    // allocation waits
    const int by_tmem = 512 / a.tmem_cols;
    smem = std::max(smem, kTcSmemSM / (by_tmem + 1) - 1024 + 256);
    smem = std::min(smem, kTcSmemMax);
    auto kern = c.C2 > 0 ? nn::conv3x3_tc_kernel<true> : nn::conv3x3_tc_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int tiles = c.N * a.tiles_y * a.tiles_x;
    kern<<<dim3(tiles, ntiles), nn::kTcThreads, smem, s>>>(map, map2, a);
    return cudaGetLastError();
}

}  // namespace lbib
