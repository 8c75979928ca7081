// sums.cu -- FP64 conservation sums of the last output step (row a7 of the
// hot path: the per-cell and global budgets that accompany the per-cell area
// of Sec. 3.3, computeAreas).
//
// One pass over the output planes of the last lbib_step() (density, velocity,
// species, labels), in the storage's compute type, accumulated in FP64:
//   global   sum rho, sum rho ux, sum rho uy, sum phi_s (every node)
//   per cell sum rho and sum phi_s over the nodes whose label (the lowest
//            cell containing the node) is the cell
//   count of nodes with a non-finite or non-positive density, a non-finite
//            velocity or a non-finite concentration
// A warp covers 32 consecutive nodes of one row.  Per-cell sums: the labels
// of a warp form runs of equal values; a segmented scan over the run gives
// its sum in the run's last lane, which adds it with one FP64 atomic.  Global
// sums: per-thread FP64 accumulators, a block reduction, one atomic per
// block and quantity.
#include <algorithm>
#include <type_traits>

#include "lbib_ctx.cuh"

namespace lbib {

constexpr int kSumThreads = 256;

template <typename C, int S>
__global__ void __launch_bounds__(kSumThreads) sums_kernel(const C* rho, const C* u,
                                                           const C* phi, const uint32_t* id,
                                                           int nx, int ny, int64_t pitch,
                                                           int64_t plane, int n_cells,
                                                           double* glob, double* cell,
                                                           unsigned* nonfinite) {
    using V2 = typename std::conditional<sizeof(C) == 8, double2, float2>::type;
    constexpr int NQ = 3 + S;  // global quantities
    double acc[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) acc[k] = 0.0;
    unsigned bad = 0u;
    const int lane = threadIdx.x & 31;
    const int warps_per_row = (nx + 31) / 32;
    const int64_t chunks = (int64_t)warps_per_row * ny;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ch = wid; ch < chunks; ch += nwarps) {
        const int y = (int)(ch / warps_per_row);
        const int x = (int)(ch - (int64_t)y * warps_per_row) * 32 + lane;
        const bool valid = x < nx;
        const int64_t node = (int64_t)y * pitch + x;
        double r = 0.0, ux = 0.0, uy = 0.0, ph[S > 0 ? S : 1];
        int c = -1;
        if (valid) {
            r = (double)rho[node];
            const V2 v = reinterpret_cast<const V2*>(u)[node];
            ux = (double)v.x;
            uy = (double)v.y;
            bool ok = r > 0.0 && isfinite(r) && isfinite(ux) && isfinite(uy);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                ph[s] = (double)phi[(int64_t)s * plane + node];
                ok = ok && isfinite(ph[s]);
            }
            if (!ok) ++bad;
            const uint32_t lab = id[node];
            if (lab != kOutside && (int)(lab >> 4) < n_cells) c = (int)(lab >> 4);
            acc[0] += r;
            acc[1] += r * ux;
            acc[2] += r * uy;
#pragma unroll
            for (int s = 0; s < S; ++s) acc[3 + s] += ph[s];
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) ph[s] = 0.0;
        }
        // runs of equal labels within the warp: the lane of a run's head and
        // the segmented inclusive scan of density and concentrations
        const int cprev = __shfl_up_sync(0xffffffffu, c, 1);
        const int cnext = __shfl_down_sync(0xffffffffu, c, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || cprev != c);
        const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
        double v[1 + (S > 0 ? S : 0)];
        v[0] = r;
#pragma unroll
        for (int s = 0; s < S; ++s) v[1 + s] = ph[s];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int k = 0; k < 1 + S; ++k) {
                const double t = __shfl_up_sync(0xffffffffu, v[k], d);
                if (lane - d >= start) v[k] += t;
            }
        }
        const bool tail = lane == 31 || cnext != c;
        if (tail && c >= 0) {
#pragma unroll
            for (int k = 0; k < 1 + S; ++k) atomicAdd(cell + (int64_t)c * (1 + S) + k, v[k]);
        }
    }
    // block reduction of the global sums
    __shared__ double red[kSumThreads / 32][NQ];
    __shared__ unsigned redbad[kSumThreads / 32];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        double t = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) red[threadIdx.x >> 5][k] = t;
    }
    const unsigned b = __reduce_add_sync(0xffffffffu, bad);
    if (lane == 0) redbad[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x < NQ) {
        double t = 0.0;
        for (int w = 0; w < kSumThreads / 32; ++w) t += red[w][threadIdx.x];
        atomicAdd(glob + threadIdx.x, t);
    }
    if (threadIdx.x == 0) {
        unsigned t = 0u;
        for (int w = 0; w < kSumThreads / 32; ++w) t += redbad[w];
        if (t) atomicAdd(nonfinite, t);
    }
}

template <typename C>
static cudaError_t launch_sums_c(int S, const lbib_ctx* c, double* glob, double* cell,
                                 unsigned* bad) {
    const Layout& L = c->L;
    const C* rho = reinterpret_cast<const C*>(c->ws + L.rho);
    const C* u = reinterpret_cast<const C*>(c->ws + L.u);
    const C* phi = reinterpret_cast<const C*>(c->ws + L.phi);
    const uint32_t* id = reinterpret_cast<const uint32_t*>(c->ws + L.id_out);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t warps = (int64_t)((c->p.nx + 31) / 32) * c->p.ny;
    const int64_t want = (warps * 32 + kSumThreads - 1) / kSumThreads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
    const int nC = c->nC;
    switch (S) {
#define LBIB_SUMS_CASE(SS)                                                                   \
    case SS:                                                                                 \
        sums_kernel<C, SS><<<grid, kSumThreads, 0, c->stream>>>(                             \
            rho, u, phi, id, c->p.nx, c->p.ny, L.pitch, L.plane, nC, glob, cell, bad);       \
        break;
        LBIB_SUMS_CASE(0)
        LBIB_SUMS_CASE(1)
        LBIB_SUMS_CASE(2)
        LBIB_SUMS_CASE(3)
        LBIB_SUMS_CASE(4)
#undef LBIB_SUMS_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbib

using namespace lbib;

extern "C" int lbib_get_sums(lbib_ctx* c, double* global_sums, double* cell_sums,
                             uint32_t* nonfinite) {
    NvtxRange nvtx_range("lbib_get_sums");
    if (!c || !global_sums) return LBIB_E_PARAM;
    if (!c->fields_valid) {
        c->err = "lbib_get_sums: the last step wrote no output fields (need lbib_step)";
        return LBIB_E_STATE;
    }
    const Layout& L = c->L;
    const int S = c->p.n_species;
    double* glob = reinterpret_cast<double*>(c->ws + L.sums);
    double* cell = glob + 4 + kMaxSpecies;
    unsigned* bad = reinterpret_cast<unsigned*>(cell + (int64_t)c->maxC * (1 + kMaxSpecies));
    const size_t cbytes = (size_t)c->nC * (1 + S) * 8;
    cudaError_t e = cudaMemsetAsync(glob, 0, L.sums_bytes, c->stream);
    if (e == cudaSuccess)
        e = c->p.precision == LBIB_FP64 ? launch_sums_c<double>(S, c, glob, cell, bad)
                                        : launch_sums_c<float>(S, c, glob, cell, bad);
    unsigned hbad = 0u;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(global_sums, glob, (size_t)(3 + S) * 8, cudaMemcpyDeviceToHost,
                            c->stream);
    if (e == cudaSuccess && cell_sums && cbytes)
        e = cudaMemcpyAsync(cell_sums, cell, cbytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("lbib_get_sums: ") + cudaGetErrorString(e);
        return LBIB_E_CUDA;
    }
    if (nonfinite) *nonfinite = hbad;
    return LBIB_OK;
}
