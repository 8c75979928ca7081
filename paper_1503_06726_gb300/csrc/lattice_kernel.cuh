// lattice_kernel.cuh -- the one-node-per-thread lattice update kernel (K1),
// included by the translation unit of the plain kernels (lattice.cu) and by
// the one of the kernels with confined species (lattice_conf.cu), which are
// compiled in parallel.
#pragma once

#include "lattice_node.cuh"

namespace lbib {

// CTAs of 128 threads.  FP32/FP16 storage is held to 40 registers with at
// most one species (12 CTAs, 48 warps per SM: more loads in flight), 48 with
// two (10 CTAs) and 64 with more (8 CTAs), none of them spilling since the
// in-plane indices are 32-bit (4096^2: 327 -> 311 us; 1024^2, two species:
// 28.6 -> 27.8 us against 48 / 56 registers).
// The kernels with confined species (CONF) hold the closure's state as well:
// 64 registers (8 CTAs per SM).
template <typename T, int S, bool CONF = false>
struct LatticeOccupancy {
    static constexpr int kMinBlocks =
        sizeof(T) == 8 ? 1 : (CONF ? 8 : (S <= 1 ? 12 : (S == 2 ? 10 : 8)));
};
constexpr int kLatticeThreads = 128;

// CONF: the paths of confined species (domain plane, no-flux closure) are
// compiled in; without it the kernel keeps the registers of the plain update
template <typename T, typename C, int S, bool WALLS, int FORCING, bool SCALED, bool CONF>
__global__ void __launch_bounds__(kLatticeThreads, LatticeOccupancy<T, S, CONF>::kMinBlocks)
    lattice_kernel(LatticeArgs a, Coefs<C> k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    constexpr bool GRIDDEP = true;
    constexpr bool OPTS = true;
    LBIB_LATTICE_NODE_BODY
}

}  // namespace lbib
