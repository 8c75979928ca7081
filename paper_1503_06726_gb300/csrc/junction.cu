// junction.cu -- renewal of the cell junctions (Eq. celljunctionforce,
// Sec. 3.2.4): every membrane point takes as partner the closest membrane
// point of another cell within l_max, or none.
//
// The vertices are put into a uniform grid of bins at least l_max wide (a
// fixed number of slots per bin; a bin that overflows raises a diagnostic
// flag and keeps its first slots), then every vertex scans the 3x3 bins
// around its own.  Distances are FP64 with the periodic minimum image in x
// (and in y without walls), evaluated with the same round-to-nearest
// operations in the same order as the definition (difference, image shift,
// squared length), so the chosen partner is that of the definition; ties go
// to the lower vertex index.  The forces themselves are added by the IB
// kernel's prep from the current positions.
#include <cmath>

#include "lbib_internal.cuh"

namespace lbib {

__device__ __forceinline__ double image_shift(double d, int n) {
    return __dsub_rn(d, __dmul_rn((double)n, round(__ddiv_rn(d, (double)n))));
}

__device__ __forceinline__ int bin_of(double X, int n, int nb, double w, bool periodic) {
    double xw = X;
    if (periodic) xw = __dsub_rn(X, __dmul_rn((double)n, floor(__ddiv_rn(X, (double)n))));
    int b = (int)floor(xw / w);
    return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__global__ void junction_bin_kernel(JunctionArgs j) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= j.nv) return;
    const double2 X = j.xy[v];
    const int bx = bin_of(X.x, j.nx, j.nbx, j.wbx, true);
    const int by = bin_of(X.y, j.ny, j.nby, j.wby, !j.bc_y);
    int* bin = j.bins + (int64_t)(by * j.nbx + bx) * (1 + kJunctionBinCap);
    const int slot = atomicAdd(bin, 1);
    if (slot < kJunctionBinCap)
        bin[1 + slot] = v;
    else
        atomicOr(j.diag + kDiagJunctionBin, 1u);
}

__global__ void junction_search_kernel(JunctionArgs j) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= j.nv) return;
    const double2 Xi = j.xy[i];
    const int ci = j.vcell[i];
    const int bx = bin_of(Xi.x, j.nx, j.nbx, j.wbx, true);
    const int by = bin_of(Xi.y, j.ny, j.nby, j.wby, !j.bc_y);
    double best = __dmul_rn(j.lmax, j.lmax);
    int bestj = -1;
    for (int dyb = -1; dyb <= 1; ++dyb) {
        int b2y = by + dyb;
        if (j.bc_y) {
            if (b2y < 0 || b2y >= j.nby) continue;
        } else {
            b2y = (b2y + j.nby) % j.nby;
        }
        for (int dxb = -1; dxb <= 1; ++dxb) {
            const int b2x = (bx + dxb + j.nbx) % j.nbx;
            const int* bin = j.bins + (int64_t)(b2y * j.nbx + b2x) * (1 + kJunctionBinCap);
            const int cnt = min(bin[0], kJunctionBinCap);
            for (int k = 0; k < cnt; ++k) {
                const int v = bin[1 + k];
                if (j.vcell[v] == ci) continue;
                const double2 Xv = j.xy[v];
                double dx = image_shift(__dsub_rn(Xv.x, Xi.x), j.nx);
                double dy = __dsub_rn(Xv.y, Xi.y);
                if (!j.bc_y) dy = image_shift(dy, j.ny);
                const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                if (d2 < best || (d2 == best && bestj >= 0 && v < bestj)) {
                    best = d2;
                    bestj = v;
                }
            }
        }
    }
    j.partner[i] = bestj;
}

cudaError_t launch_junction_renew(const JunctionArgs& j, cudaStream_t s) {
    if (j.nv <= 0) return cudaSuccess;
    // bin counts to zero: the first int of every bin
    cudaError_t e = cudaMemset2DAsync(j.bins, (size_t)(1 + kJunctionBinCap) * 4, 0, 4,
                                      (size_t)j.nbx * j.nby, s);
    if (e != cudaSuccess) return e;
    const int threads = 256, blocks = (j.nv + threads - 1) / threads;
    e = launch_kernel(junction_bin_kernel, dim3(blocks), dim3(threads), 0, s, false, j);
    if (e != cudaSuccess) return e;
    return launch_kernel(junction_search_kernel, dim3(blocks), dim3(threads), 0, s, false, j);
}

}  // namespace lbib
