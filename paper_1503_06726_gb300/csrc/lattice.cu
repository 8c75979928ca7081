// lattice.cu -- the fused lattice update of one coupled step (K1).
//
// One thread per lattice node, pull scheme: the kernel streams the
// post-collision populations of the previous step from the neighbours
// (left-hand side of Eq. bgkequation, Sec. 6.1), forms the moments, collides
// the D2Q9 fluid with the BGK operator and the body force, and updates every
// D2Q5 species with the same velocity and its reaction term, writing the new
// post-collision populations to the other buffer.  The spread IB force and
// the cell labels of the node are read and reset to their empty values in
// the same pass, so no separate clearing pass is needed.
//
// Storage is SoA: one plane per population, rows of `pitch` elements, plane
// q at q*plane.  Populations are stored as deviations from the rest state,
// d_q = f_q - w_q rho0 (species: g_q itself), optionally scaled for FP16
// (stored = d_q / (w_q sigma)).  The collision is evaluated in deviation
// space, which keeps FP32/FP16 storage accurate:
//   rho = rho0 + sum d,  rho u = sum d v (+ F/2 for Guo forcing)
//   d_eq = w (drho + rho (3 v.u + 9/2 (v.u)^2 - 3/2 u.u))   (Eq. standardequilibrium)
//   d*   = d + (d_eq - d)/tau + S_q                       (Eq. bgkequation)
// with S_q the Guo source (1 - 1/(2 tau)) w [3 (v - u) + 9 (v.u) v].F or the
// paper's 3 w v.F.  Species (D2Q5): phi = sum g, g_eq = phi w (1 + 3 v.u),
// g* = g + (g_eq - g)/tau_D + w R with R the linear reaction plus the source
// of the node's cell.
#include <type_traits>

#include "lattice_node.cuh"

namespace lbib {

// CTAs of 128 threads.  FP32/FP16 storage is held to 48 registers with one
// species (10 CTAs, 40 warps per SM: more loads in flight, measured faster),
// 56 with two (9 CTAs; 48 spilled) and 64 with more (8 CTAs, no spills).
template <typename T, int S>
struct LatticeOccupancy {
    static constexpr int kMinBlocks = sizeof(T) == 8 ? 1 : (S <= 1 ? 10 : (S == 2 ? 9 : 8));
};
constexpr int kLatticeThreads = 128;

template <typename T, typename C, int S, bool WALLS, int FORCING, bool SCALED>
__global__ void __launch_bounds__(kLatticeThreads, LatticeOccupancy<T, S>::kMinBlocks)
    lattice_kernel(LatticeArgs a, Coefs<C> k) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    constexpr bool GRIDDEP = true;
    LBIB_LATTICE_NODE_BODY
}

template <typename T, typename C, int S, bool WALLS, int FORCING>
static cudaError_t launch3(const LatticeArgs& a, const void* coefs, dim3 block, cudaStream_t s,
                           bool pdl) {
    // the group masks are cleared per warp: a warp must be 32 nodes of one row
    if (a.fmask && block.x % 32 != 0) return cudaErrorInvalidConfiguration;
    if (block.x * block.y * block.z > (unsigned)kLatticeThreads) return cudaErrorInvalidConfiguration;
    dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
    const Coefs<C>& k = *static_cast<const Coefs<C>*>(coefs);
    constexpr bool SC = std::is_same<T, __half>::value;
    return launch_kernel(lattice_kernel<T, C, S, WALLS, FORCING, SC>, grid, block, 0, s, pdl, a,
                         k);
}

template <typename T, typename C, int S>
static cudaError_t launch2(int bc_y, int forcing, const LatticeArgs& a, const void* coefs,
                           dim3 block, cudaStream_t s, bool pdl) {
    if (bc_y) {
        return forcing ? launch3<T, C, S, true, 1>(a, coefs, block, s, pdl)
                       : launch3<T, C, S, true, 0>(a, coefs, block, s, pdl);
    }
    return forcing ? launch3<T, C, S, false, 1>(a, coefs, block, s, pdl)
                   : launch3<T, C, S, false, 0>(a, coefs, block, s, pdl);
}

template <typename T, typename C>
static cudaError_t launch1(int n_species, int bc_y, int forcing, const LatticeArgs& a,
                           const void* coefs, dim3 block, cudaStream_t s, bool pdl) {
    switch (n_species) {
        case 0: return launch2<T, C, 0>(bc_y, forcing, a, coefs, block, s, pdl);
        case 1: return launch2<T, C, 1>(bc_y, forcing, a, coefs, block, s, pdl);
        case 2: return launch2<T, C, 2>(bc_y, forcing, a, coefs, block, s, pdl);
        case 3: return launch2<T, C, 3>(bc_y, forcing, a, coefs, block, s, pdl);
        default: return launch2<T, C, 4>(bc_y, forcing, a, coefs, block, s, pdl);
    }
}

cudaError_t launch_lattice(int precision, int n_species, int bc_y, int forcing,
                           const LatticeArgs& a, const void* coefs, dim3 block, cudaStream_t s,
                           bool pdl) {
    if (precision == LBIB_FP64)
        return launch1<double, double>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
    if (precision == LBIB_FP32)
        return launch1<float, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
    return launch1<__half, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
}

// ---------------------------------------------------------------------------
// rest state: d = 0 (f = w rho0), g = 0 -- all stored values are zero
template <typename T>
__global__ void zero_planes(T* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += st) p[i] = T(0);
}

cudaError_t launch_init_populations(int precision, int n_species, int nx, int ny, int64_t pitch,
                                    int64_t plane, void* f, void* g, cudaStream_t s) {
    (void)nx; (void)ny; (void)pitch; (void)precision;
    // every storage type represents zero with all-zero bytes
    int es = precision == LBIB_FP64 ? 8 : (precision == LBIB_FP32 ? 4 : 2);
    cudaError_t e = cudaMemsetAsync(f, 0, (size_t)9 * plane * es, s);
    if (e != cudaSuccess) return e;
    if (n_species > 0) e = cudaMemsetAsync(g, 0, (size_t)5 * n_species * plane * es, s);
    return e;
}

template <typename T, typename C>
__global__ void set_species_kernel(int nx, int ny, int64_t pitch, int64_t plane,
                                   const double* phi, T* g, Coefs<C> k, bool scaled) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= nx || y >= ny) return;
    double v = phi[(int64_t)y * nx + x];
    for (int q = 0; q < 5; ++q) {
        C gq = C(w5(q) * v);
        if (scaled) gq *= k.ginv[q];
        Store<T, C>::st(g + q * plane + (int64_t)y * pitch + x, gq);
    }
}

cudaError_t launch_set_species(int precision, int n_species, int s_idx, int nx, int ny,
                               int64_t pitch, int64_t plane, const double* phi, void* g,
                               const void* coefs, cudaStream_t s) {
    (void)n_species;
    dim3 block(128), grid((nx + 127) / 128, ny);
    if (precision == LBIB_FP64) {
        set_species_kernel<double, double><<<grid, block, 0, s>>>(
            nx, ny, pitch, plane, phi, static_cast<double*>(g) + (int64_t)s_idx * 5 * plane,
            *static_cast<const Coefs<double>*>(coefs), false);
    } else if (precision == LBIB_FP32) {
        set_species_kernel<float, float><<<grid, block, 0, s>>>(
            nx, ny, pitch, plane, phi, static_cast<float*>(g) + (int64_t)s_idx * 5 * plane,
            *static_cast<const Coefs<float>*>(coefs), false);
    } else {
        set_species_kernel<__half, float><<<grid, block, 0, s>>>(
            nx, ny, pitch, plane, phi, static_cast<__half*>(g) + (int64_t)s_idx * 5 * plane,
            *static_cast<const Coefs<float>*>(coefs), true);
    }
    return cudaGetLastError();
}

}  // namespace lbib
