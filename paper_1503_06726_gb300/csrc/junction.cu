// junction.cu -- renewal of the cell junctions (Eq. celljunctionforce,
// Sec. 3.2.4): every membrane point takes as partner the closest membrane
// point of another cell within l_max, or none.
//
// The vertices are sorted into a uniform grid of bins at least l_max wide
// (CSR: count, one-CTA scan, fill; no per-bin capacity), then every vertex
// scans the 3x3 bins around its own with a group of lanes that share its
// candidates.  Each candidate first passes an FP32
// test on wrapped positions whose bound exceeds l_max by more than the FP32
// rounding can move a distance, so it only drops vertices that are certainly
// out of range; the survivors take the definition's FP64 test (difference,
// periodic minimum image, squared length, round-to-nearest in that order), so
// the chosen partner is that of the definition; ties go to the lower vertex
// index.  The forces themselves are added by the IB kernel's prep from the
// current positions.
#include <cmath>

#include "lbib_internal.cuh"

namespace lbib {

// Bin of coordinate X on an axis of n nodes cut into nb bins of width w (the
// coordinate wrapped into [0, n) on a periodic axis, clamped to the end bins
// on a walled one).  Every vertex's bin is computed once and stored, so the
// multiplications by reciprocals only have to keep the bins at least l_max
// wide, which the 1e-4 margin of the width covers.
__device__ __forceinline__ int bin_axis(double X, int n, double inv_n, int nb, double inv_w,
                                        bool periodic, double* wrapped) {
    double xw = X;
    if (periodic) xw = X - (double)n * floor(X * inv_n);
    *wrapped = xw;
    const int b = (int)floor(xw * inv_w);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__device__ __forceinline__ int vertex_bin(const JunctionArgs& j, double2 X, float2* wrapped) {
    double xw, yw;
    const int bx = bin_axis(X.x, j.nx, j.inv_nx, j.nbx, j.inv_wbx, true, &xw);
    const int by = bin_axis(X.y, j.ny, j.inv_ny, j.nby, j.inv_wby, !j.bc_y, &yw);
    *wrapped = make_float2((float)xw, (float)yw);
    return by * j.nbx + bx;
}

__global__ void junction_count_kernel(JunctionArgs j) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= j.nv) return;
    float2 w;
    const int b = vertex_bin(j, j.xy[v], &w);
    j.vbin[v] = b;
    atomicAdd(j.cnt + b, 1);
}

// exclusive scan of the bin counts into start[0..nbins] (one CTA of 1024
// threads, a contiguous run of bins per thread); the counts become the fill
// cursors
__global__ void __launch_bounds__(1024) junction_scan_kernel(JunctionArgs j) {
    __shared__ int wsum[32];
    const int nb = j.nbx * j.nby;
    const int per = (nb + 1023) / 1024;
    const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += j.cnt[b];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    int excl = x - s + (w > 0 ? wsum[w - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const int c = j.cnt[b];
        j.start[b] = excl;
        j.cnt[b] = excl;
        excl += c;
    }
    if (threadIdx.x == 1023) j.start[nb] = excl;  // the last thread ends at the total
}

__global__ void junction_fill_kernel(JunctionArgs j) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= j.nv) return;
    float2 w;
    vertex_bin(j, j.xy[v], &w);
    const int slot = atomicAdd(j.cnt + j.vbin[v], 1);
    JunctionEntry e;
    e.x = w.x;
    e.y = w.y;
    e.cell = j.vcell[v];
    e.v = v;
    j.ent[slot] = e;
}

__device__ __forceinline__ float fold(float d, float n, float half) {
    return d > half ? d - n : (d < -half ? d + n : d);
}

// lanes that share one vertex's candidates (an aligned group within a warp)
constexpr int kSearchLanes = 8;

__global__ void junction_search_kernel(JunctionArgs j) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gt / kSearchLanes);
    const int r = (int)(gt % kSearchLanes);
    double best = __dmul_rn(j.lmax, j.lmax);
    int bestj = -1;
    if (i < j.nv) {
        const double2 Xi = j.xy[i];
        const int ci = j.vcell[i];
        float2 wi;
        vertex_bin(j, Xi, &wi);
        const int b = j.vbin[i];
        const int bx = b % j.nbx, by = b / j.nbx;
        const float nxf = (float)j.nx, nyf = (float)j.ny;
        const float hx = 0.5f * nxf, hy = 0.5f * nyf;
        for (int dyb = -1; dyb <= 1; ++dyb) {
            int b2y = by + dyb;
            if (j.bc_y) {
                if (b2y < 0 || b2y >= j.nby) continue;
            } else {
                b2y = (b2y + j.nby) % j.nby;
            }
            for (int dxb = -1; dxb <= 1; ++dxb) {
                const int b2 = b2y * j.nbx + (bx + dxb + j.nbx) % j.nbx;
                const int s1 = j.start[b2 + 1];
                for (int s = j.start[b2] + r; s < s1; s += kSearchLanes) {
                    const JunctionEntry e = j.ent[s];
                    if (e.cell == ci) continue;
                    const float fx = fold(e.x - wi.x, nxf, hx);
                    const float fy = j.bc_y ? e.y - wi.y : fold(e.y - wi.y, nyf, hy);
                    if (fx * fx + fy * fy > j.fthr) continue;
                    // the definition's test in FP64
                    const double2 Xv = j.xy[e.v];
                    const double dx = min_image(__dsub_rn(Xv.x, Xi.x), j.nx);
                    double dy = __dsub_rn(Xv.y, Xi.y);
                    if (!j.bc_y) dy = min_image(dy, j.ny);
                    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                    if (d2 < best || (d2 == best && bestj >= 0 && e.v < bestj)) {
                        best = d2;
                        bestj = e.v;
                    }
                }
            }
        }
    }
    // the closest candidate over the vertex's lanes, ties to the lower index
    // (a found candidate is always strictly closer than l_max, so "none"
    // never ties with one)
#pragma unroll
    for (int o = kSearchLanes / 2; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bestj, o);
        if (ob < best || (ob == best && oj >= 0 && (bestj < 0 || oj < bestj))) {
            best = ob;
            bestj = oj;
        }
    }
    if (i < j.nv && r == 0) j.partner[i] = bestj;
}

cudaError_t launch_junction_renew(const JunctionArgs& j, cudaStream_t s) {
    if (j.nv <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(j.cnt, 0, (size_t)j.nbx * j.nby * 4, s);
    if (e != cudaSuccess) return e;
    const int threads = 256, blocks = (j.nv + threads - 1) / threads;
    e = launch_kernel(junction_count_kernel, dim3(blocks), dim3(threads), 0, s, false, j);
    if (e == cudaSuccess)
        e = launch_kernel(junction_scan_kernel, dim3(1), dim3(1024), 0, s, false, j);
    if (e == cudaSuccess)
        e = launch_kernel(junction_fill_kernel, dim3(blocks), dim3(threads), 0, s, false, j);
    // kSearchLanes lanes per vertex; the block size keeps every group of
    // lanes inside one warp
    const int64_t search_blocks = ((int64_t)j.nv * kSearchLanes + threads - 1) / threads;
    if (e == cudaSuccess)
        e = launch_kernel(junction_search_kernel, dim3((unsigned)search_blocks), dim3(threads), 0,
                          s, false, j);
    return e;
}

}  // namespace lbib
