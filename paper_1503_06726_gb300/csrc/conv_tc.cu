// conv_tc.cu -- the 3x3 convolutions of the neural operator on the fifth-
// generation tensor cores: tcgen05.mma (BF16 operands, FP32 accumulation)
// with the accumulator in tensor memory (TMEM), operands staged in shared
// memory by the tensor memory accelerator (TMA), one thread issuing the
// matrix multiplies, mbarriers pacing two pipeline stages.
//
// Implicit GEMM: M = output pixels, N = all output channels (rounded up to
// 16; more than 192 split into equal tiles of at most 192, one per CTA
// column of the grid), K = 9 taps x input channels, in chunks of 16.  A tap
// (ky, kx) reads the pixel tile shifted by (ky - 1, kx - 1), and its A
// operand must be a K-major matrix whose rows (one per output pixel) lie 16
// bytes apart -- the canonical layout without swizzling (core matrices of 8
// rows x 16 bytes; the two 8-channel halves of a chunk a fixed offset
// apart).  Two tile shapes make every tap such a window of the staged halo:
//   wide images (W a multiple of 128): a CTA takes m image rows of 128
//   pixels, one accumulator of 128 TMEM lanes per row; the halo holds
//   (m + 2) rows of 130 pixels, and row j's tap (ky, kx) starts at halo row
//   j + ky, column kx -- one 4-D TMA box (8 channels x 130 x (m + 2) x 1)
//   per 8-channel half;
//   narrow images (W = 16, 32, 64): a CTA takes R = 128 / W whole rows in
//   one accumulator; the halo is staged three times, copy kx holding columns
//   kx - 1 .. kx + W - 2, so that tap (ky, kx) is copy kx from row ky on --
//   one TMA box (8 x W x (R + 2) x 1) per copy and half.
// The image's zero padding is the TMA's out-of-bounds fill.  The decoder's
// upsampled half-resolution channels (each value repeated 2 x 2) are staged
// by the threads with cp.async instead.  The weights are pre-tiled
// (tile_weights_tc_kernel) into the order the B descriptors read, [N tile]
// [chunk][tap][half][output channel][8 input channels], so that one bulk
// copy loads a chunk's weights for all nine taps.  Chunks stream through
// two or three stages of shared memory.
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

constexpr int kTcThreads = 128;  // four warps: the accumulator's four lane quarters
constexpr int kTcM = 128;
constexpr int kTcChunk = 16;     // input channels per K chunk (one MMA per tap)

struct ConvTcArgs {
    const __nv_bfloat16* in2;  // (N, H/2, W/2, C2), read upsampled, or NULL
    const __nv_bfloat16* wt;   // tiled weights, [N tiles][nk][9][2][Np][8]
    const float* bias;         // (Co) or NULL
    void* out;                 // (N, H, W, Co) bf16, or fp32 when out_f32
    unsigned* err;             // raised when a bounded wait runs out
    int N, H, W, C1, C2, Co, nk;
    int Np;                    // output channels of one CTA (N tile)
    int Wt, R, m;              // tile: m accumulators of R rows x Wt pixels (R * Wt = 128)
    int wide;                  // 1: one halo of rows of Wt + 2 pixels; 0: three kx copies
    int rs;                    // halo row stride in pixels (Wt + 2, or Wt)
    int nc;                    // halo copies (1, or 3)
    int relu, out_f32;
    int box_bytes;             // one halo copy of one 8-channel half: (m R + 2) rs 16
    int copy_bytes;            // box_bytes rounded up to 128 (TMA destinations)
    int stage_bytes;           // A and B of one chunk, rounded up to 1024
    int stages;                // 2 or 3
    int tmem_cols;             // power of two >= max(32, m Np)
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
// Shared memory matrix descriptor, K-major without swizzling: start address,
// the byte distance between the two 16-byte K core matrices of an MMA (lbo)
// and between consecutive groups of 8 rows (sbo), all in 16-byte units; bits
// 46-47 hold the descriptor version of this architecture (1).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
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

constexpr int kTcMaxStages = 3;

__global__ void __launch_bounds__(kTcThreads, 1)
    conv3x3_tc_kernel(const __grid_constant__ CUtensorMap map1, ConvTcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kTcMaxStages], bar_done[kTcMaxStages];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_bad, s_committed;
    // stages at 1024-byte boundaries (TMA destinations need 128)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = a.stages;

    const int TR = a.m * a.R;  // image rows of the tile
    const int tiles_x = a.W / a.Wt, tiles_y = a.H / TR;
    const int n = blockIdx.x / (tiles_x * tiles_y);
    const int rem = blockIdx.x % (tiles_x * tiles_y);
    const int y0 = (rem / tiles_x) * TR, x0 = (rem % tiles_x) * a.Wt;
    const int co0 = blockIdx.y * a.Np;  // this CTA's output channels
    const __nv_bfloat16* wt = a.wt + (int64_t)blockIdx.y * a.nk * 9 * 2 * a.Np * 8;

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
    const int a_bytes = 2 * a.nc * a.copy_bytes;
    const uint32_t b_bytes = 18u * (uint32_t)a.Np * 16u;
    const int hrows = TR + 2;
    // thread 0: the chunk whose loads were issued into a stage and not yet
    // waited for (-1 = none)
    int loading[kTcMaxStages] = {-1, -1, -1};

    for (int k = 0; k < a.nk; ++k) {
        const int s = k % NS;
        const uint32_t st = base + (uint32_t)s * (uint32_t)a.stage_bytes;
        // the stage was read by the multiplies of chunk k - NS
        if (k >= NS && !mbar_wait(smem_u32(&bar_done[s]), ((k - NS) / NS) & 1)) s_bad = 1;
        __syncthreads();
        if (s_bad) break;
        const int c0 = k * kTcChunk;
        const bool from1 = c0 < a.C1;
        if (tid == 0) {
            const uint32_t fb = smem_u32(&bar_full[s]);
            mbar_expect_tx(fb, b_bytes + (from1 ? (uint32_t)(2 * a.nc * a.box_bytes) : 0u));
            if (from1) {
                for (int h = 0; h < 2; ++h)
                    for (int cp = 0; cp < a.nc; ++cp)
                        tma_load_4d(st + (uint32_t)((h * a.nc + cp) * a.copy_bytes), &map1,
                                    c0 + 8 * h, a.wide ? x0 - 1 : x0 + cp - 1, y0 - 1, n, fb);
            }
            bulk_load(st + (uint32_t)a_bytes, wt + (int64_t)k * 9 * 2 * a.Np * 8, b_bytes, fb);
            loading[s] = k;
        }
        if (!from1) {
            // upsampled half-resolution channels: every thread stages 16-byte
            // pieces (8 channels of one halo pixel), zeros outside the image
            const int cc = c0 - a.C1;
            const int per_copy = hrows * a.rs;
            for (int i = tid; i < 2 * a.nc * per_copy; i += kTcThreads) {
                const int cp = i / per_copy, hp = i % per_copy;
                const int h = cp / a.nc, kx = cp % a.nc;
                const int gy = y0 + hp / a.rs - 1;
                const int gx = x0 + hp % a.rs - 1 + (a.wide ? 0 : kx);
                const bool ok = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
                const __nv_bfloat16* src =
                    ok ? a.in2 + (((int64_t)n * (a.H >> 1) + (gy >> 1)) * (a.W >> 1) + (gx >> 1)) *
                                     a.C2 + cc + 8 * h
                       : a.in2;
                cp_async16_zfill(st + (uint32_t)(cp * a.copy_bytes + hp * 16), src, ok);
            }
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
            // written through the generic proxy, read by the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            if (!mbar_wait(smem_u32(&bar_full[s]), (k / NS) & 1)) {
                s_bad = 1;
            } else {
                loading[s] = -1;
                tc_fence_after();
                const uint32_t lbo = (uint32_t)(a.nc * a.copy_bytes);
                for (int t = 0; t < 9; ++t) {
                    const int ky = t / 3, kx = t % 3;
                    const uint32_t bad = st + (uint32_t)a_bytes + (uint32_t)(t * 2 * a.Np * 16);
                    const uint64_t bdesc = smem_desc(bad, (uint32_t)a.Np * 16u, 128u);
                    for (int j = 0; j < a.m; ++j) {
                        const int row = j * a.R + ky;
                        const uint32_t aad =
                            st + (uint32_t)((a.wide ? 0 : kx) * a.copy_bytes) +
                            (uint32_t)((row * a.rs + (a.wide ? kx : 0)) * 16);
                        tc_mma(tmem + (uint32_t)(j * a.Np), smem_desc(aad, lbo, 128u), bdesc,
                               idesc, (k > 0 || t > 0) ? 1u : 0u);
                    }
                }
                tc_commit(smem_u32(&bar_done[s]));
                s_committed = k;
            }
        }
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
        const int p = warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int j = 0; j < a.m; ++j) {
            const int gy = y0 + j * a.R + p / a.Wt, gx = x0 + p % a.Wt;
            const int64_t pix = ((int64_t)n * a.H + gy) * a.W + gx;
            for (int cl = 0; cl < a.Np; cl += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)(j * a.Np + cl), v);
                const int c0 = co0 + cl;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int co = c0 + i;
                    if (co < a.Co) {
                        if (a.bias) v[i] += a.bias[co];
                        if (a.relu) v[i] = fmaxf(v[i], 0.f);
                    }
                }
                if (a.out_f32) {
                    float* o = static_cast<float*>(a.out) + pix * a.Co;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < a.Co) o[c0 + i] = v[i];
                } else {
                    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.out) + pix * a.Co + c0;
                    if (c0 + 16 <= a.Co && (a.Co % 8) == 0) {
                        uint4 w0, w1;
                        __nv_bfloat162 h[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                        std::memcpy(&w0, &h[0], 16);
                        std::memcpy(&w1, &h[4], 16);
                        reinterpret_cast<uint4*>(o)[0] = w0;
                        reinterpret_cast<uint4*>(o)[1] = w1;
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < a.Co) o[i] = __float2bfloat16_rn(v[i]);
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

// Weights (9, Co, Ci) -> [N tiles][Ci/16 chunks][9 taps][2 halves][Np][8]
// (Np output channels per tile), zeros for output channels >= Co and input
// channels >= Ci.
__global__ void tile_weights_tc_kernel(const __nv_bfloat16* w, int Co, int Ci, int Np, int nk,
                                       int ntiles, __nv_bfloat16* wt) {
    const int64_t per_tile = (int64_t)nk * 9 * 2 * Np * 8;
    const int64_t total = per_tile * ntiles;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i % per_tile;
        const int tile = (int)(i / per_tile);
        const int j = (int)(r % 8);
        const int co = tile * Np + (int)((r / 8) % Np);
        const int h = (int)((r / (8 * Np)) % 2);
        const int t = (int)((r / (16 * Np)) % 9);
        const int k = (int)(r / (144 * (int64_t)Np));
        const int ci = k * kTcChunk + 8 * h + j;
        wt[i] = (co < Co && ci < Ci) ? w[((int64_t)t * Co + co) * Ci + ci] : __float2bfloat16(0.f);
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

// pixel tile of an H x W image: R rows of Wt pixels, R * Wt = 128
static bool tc_tile(int H, int W, int* R, int* Wt) {
    if (W >= 128) {
        if (W % 128) return false;
        *Wt = 128;
        *R = 1;
    } else {
        if (W < 16 || 128 % W) return false;
        *Wt = W;
        *R = 128 / W;
    }
    return H % *R == 0;
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

// The tile plan: m accumulators per CTA -- the largest of 4, 2, 1 that
// divides the image rows, fits TMEM (m Np <= 512 columns) and two stages of
// shared memory, and still leaves two CTAs per SM -- and three stages where
// they fit.
static bool tc_plan(int N, int H, int W, int Np, int ntiles, nn::ConvTcArgs* a) {
    int R, Wt;
    if (!tc_tile(H, W, &R, &Wt)) return false;
    a->R = R;
    a->Wt = Wt;
    a->wide = Wt == 128 ? 1 : 0;
    a->rs = a->wide ? Wt + 2 : Wt;
    a->nc = a->wide ? 1 : 3;
    for (int m = 4; m >= 1; m /= 2) {
        if (H % (m * R) || m * Np > 512) continue;
        const int64_t ctas = (int64_t)N * (H / (m * R)) * (W / Wt) * ntiles;
        if (m > 1 && ctas < 2 * sm_count()) continue;
        const int box = (m * R + 2) * a->rs * 16;
        const int copy = (box + 127) / 128 * 128;
        const int stage = (2 * a->nc * copy + 18 * Np * 16 + 1023) / 1024 * 1024;
        if (2 * stage + 1024 > kTcSmemMax) continue;
        a->m = m;
        a->box_bytes = box;
        a->copy_bytes = copy;
        a->stage_bytes = stage;
        a->stages = 3 * stage + 1024 <= kTcSmemMax ? 3 : 2;
        a->tmem_cols = 32;
        while (a->tmem_cols < m * Np) a->tmem_cols *= 2;
        return true;
    }
    return false;
}

// output channels per CTA: all of them (rounded up to 16) up to 192, else
// equal tiles of at most 192
static void tc_ntiles(int Co, int* ntiles, int* Np) {
    const int n16 = (Co + 15) / 16;
    *ntiles = (n16 + 11) / 12;
    *Np = (n16 + *ntiles - 1) / *ntiles * 16;
}

int64_t tc_tiled_weight_elems(int Ci, int Co) {
    int nt, Np;
    tc_ntiles(Co, &nt, &Np);
    return (int64_t)nt * ((Ci + nn::kTcChunk - 1) / nn::kTcChunk) * 9 * 2 * Np * 8;
}

bool tc_conv_supported(int H, int W, int C1, int C2, int Co) {
    int R, Wt;
    return tc_tile(H, W, &R, &Wt) && C1 >= 16 && C1 % 16 == 0 && C2 % 16 == 0 && Co >= 1 &&
           (C2 == 0 || (H % 2 == 0 && W % 2 == 0)) && encode_fn() != nullptr;
}

cudaError_t tc_tile_weights(const void* w, int Co, int Ci, void* wt, cudaStream_t s) {
    int nt, Np;
    tc_ntiles(Co, &nt, &Np);
    const int nk = (Ci + nn::kTcChunk - 1) / nn::kTcChunk;
    const int64_t total = (int64_t)nt * nk * 9 * 2 * Np * 8;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 4096);
    nn::tile_weights_tc_kernel<<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(w), Co, Ci,
                                                      Np, nk, nt, static_cast<__nv_bfloat16*>(wt));
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
    a.err = err;
    a.N = c.N;
    a.H = c.H;
    a.W = c.W;
    a.C1 = c.C1;
    a.C2 = c.C2;
    a.Co = c.Co;
    int ntiles = 1;
    tc_ntiles(c.Co, &ntiles, &a.Np);
    if (!tc_plan(c.N, c.H, c.W, a.Np, ntiles, &a)) return cudaErrorInvalidValue;
    a.nk = (c.C1 + c.C2) / nn::kTcChunk;
    a.relu = c.relu;
    a.out_f32 = c.out_f32;
    // the full-resolution input as a 4-D tensor (channels, x, y, image); one
    // box is 8 channels x rs pixels x (m R + 2) rows of one image
    CUtensorMap map;
    std::memset(&map, 0, sizeof(map));
    cuuint64_t dims[4] = {(cuuint64_t)c.C1, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
    cuuint64_t strides[3] = {(cuuint64_t)c.C1 * 2, (cuuint64_t)c.W * c.C1 * 2,
                             (cuuint64_t)c.H * c.W * c.C1 * 2};
    cuuint32_t box[4] = {8, (cuuint32_t)a.rs, (cuuint32_t)(a.m * a.R + 2), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
                             const_cast<__nv_bfloat16*>(c.in1), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    int smem = a.stages * a.stage_bytes + 1024;
    // more than half of TMEM: one CTA per SM, so that no allocation waits
    if (a.tmem_cols > 256) smem = std::max(smem, 120 * 1024);
    cudaError_t e = cudaFuncSetAttribute(nn::conv3x3_tc_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int tiles = c.N * (c.H / (a.m * a.R)) * (c.W / a.Wt);
    nn::conv3x3_tc_kernel<<<dim3(tiles, ntiles), nn::kTcThreads, smem, s>>>(map, a);
    return cudaGetLastError();
}

}  // namespace lbib
