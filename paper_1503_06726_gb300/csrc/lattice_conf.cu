// lattice_conf.cu -- the lattice update with confined species, and the set-up
// of the membrane no-flux closure (Sec. 6.1, no-flux boundary condition for
// reaction-advection-diffusion equations).
//
// A confined species does not take a population that would arrive at a node
// x along v_q from a node of another domain (the static label plane of
// lbib_set_domains).  The paper replaces such a missing population by an
// equilibrium whose momentum is interpolated to first order between the fluid
// in the direction of the missing population and zero at the wall, and whose
// density is extrapolated to first order from the fluid.  Here the wall point
// is the half-way point of the crossing link, the fluid nodes are
// y1 = x + v_q and y2 = x + 2 v_q, and their densities and momenta (first
// moments of the species) are those of the previous step: the missing
// population is w_q (2 phi(y1) - phi(y2) + v_q . j(y1)) (pull5_closure).
// Which links cross a membrane and which of y1, y2 lie in the domain depend
// on the labels only, so they are coded once per node (make_ncode_kernel);
// the lattice kernel reads one 16-bit code per node, and writes its species
// moments only where a closure of the next step reads them.  With
// noflux_scheme 1 the kernels reflect the population instead (half-way
// bounce-back, exact per-domain mass; not the paper's condition).
#include "lattice_kernel.cuh"

namespace lbib {

template <typename T, typename C, int S, bool WALLS, int FORCING>
static cudaError_t launch_conf3(const LatticeArgs& a, const void* coefs, dim3 block,
                                cudaStream_t s, bool pdl) {
    if (a.fmask && block.x % 32 != 0) return cudaErrorInvalidConfiguration;
    if (block.x * block.y * block.z > (unsigned)kLatticeThreads) return cudaErrorInvalidConfiguration;
    // the closure needs its moment planes
    if (a.ncode && (!a.mom_in || !a.mom_out)) return cudaErrorInvalidValue;
    dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
    const Coefs<C>& k = *static_cast<const Coefs<C>*>(coefs);
    constexpr bool SC = std::is_same<T, __half>::value;
    return launch_kernel(lattice_kernel<T, C, S, WALLS, FORCING, SC, true>, grid, block, 0, s,
                         pdl, a, k);
}

template <typename T, typename C, int S>
static cudaError_t launch_conf2(int bc_y, int forcing, const LatticeArgs& a, const void* coefs,
                                dim3 block, cudaStream_t s, bool pdl) {
    if (bc_y)
        return forcing ? launch_conf3<T, C, S, true, 1>(a, coefs, block, s, pdl)
                       : launch_conf3<T, C, S, true, 0>(a, coefs, block, s, pdl);
    return forcing ? launch_conf3<T, C, S, false, 1>(a, coefs, block, s, pdl)
                   : launch_conf3<T, C, S, false, 0>(a, coefs, block, s, pdl);
}

template <typename T, typename C>
static cudaError_t launch_conf1(int n_species, int bc_y, int forcing, const LatticeArgs& a,
                                const void* coefs, dim3 block, cudaStream_t s, bool pdl) {
    switch (n_species) {
        case 1: return launch_conf2<T, C, 1>(bc_y, forcing, a, coefs, block, s, pdl);
        case 2: return launch_conf2<T, C, 2>(bc_y, forcing, a, coefs, block, s, pdl);
        case 3: return launch_conf2<T, C, 3>(bc_y, forcing, a, coefs, block, s, pdl);
        case 4: return launch_conf2<T, C, 4>(bc_y, forcing, a, coefs, block, s, pdl);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lattice_confined(int precision, int n_species, int bc_y, int forcing,
                                    const LatticeArgs& a, const void* coefs, dim3 block,
                                    cudaStream_t s, bool pdl) {
    if (precision == LBIB_FP64)
        return launch_conf1<double, double>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
    if (precision == LBIB_FP32)
        return launch_conf1<float, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
    return launch_conf1<__half, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl);
}

// ---------------------------------------------------------------------------
// The closure codes.  Node (i, j) of the lattice; a label beyond a wall does
// not exist (lab_at returns false).
__device__ __forceinline__ bool lab_at(const int32_t* dom, int i, int j, int nx, int ny,
                                       int bc_y, int64_t pitch, int32_t* out) {
    if (j < 0 || j >= ny) {
        if (bc_y) return false;
        j = j < 0 ? j + ny : j - ny;
    }
    i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
    *out = dom[(int64_t)j * pitch + i];
    return true;
}

// bits kNcodeMiss, kNcodeIn1, kNcodeIn2 of node (i, j)
__device__ uint32_t ncode_links(const int32_t* dom, int i, int j, int nx, int ny, int bc_y,
                                int64_t pitch) {
    int32_t d0;
    lab_at(dom, i, j, nx, ny, bc_y, pitch, &d0);
    uint32_t code = 0u;
#pragma unroll
    for (int q = 1; q <= 4; ++q) {
        const int vx = cx(q), vy = cy(q);
        int32_t ds, d1, d2;
        // the population arriving along v_q left i - v_q: a membrane when that
        // node exists (a wall link reflects) and lies in another domain
        if (lab_at(dom, i - vx, j - vy, nx, ny, bc_y, pitch, &ds) && ds != d0)
            code |= 1u << (kNcodeMiss + q - 1);
        const bool in1 = lab_at(dom, i + vx, j + vy, nx, ny, bc_y, pitch, &d1) && d1 == d0;
        const bool in2 =
            in1 && lab_at(dom, i + 2 * vx, j + 2 * vy, nx, ny, bc_y, pitch, &d2) && d2 == d0;
        if (in1) code |= 1u << (kNcodeIn1 + q - 1);
        if (in2) code |= 1u << (kNcodeIn2 + q - 1);
    }
    return code;
}

// Every node's code, with kNcodeMom where a closure reads the node's moments:
// the node is y1 of the closure of x = node - v_q, y2 of the one of
// x = node - 2 v_q, or (no fluid node along the link) x itself.
__global__ void make_ncode_kernel(const int32_t* dom, uint16_t* ncode, int nx, int ny, int bc_y,
                                  int64_t pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= nx || j >= ny) return;
    uint32_t code = ncode_links(dom, i, j, nx, ny, bc_y, pitch);
    bool mom = false;
#pragma unroll
    for (int q = 1; q <= 4; ++q) {
        const int vx = cx(q), vy = cy(q);
        const uint32_t miss = 1u << (kNcodeMiss + q - 1);
        const uint32_t in1 = 1u << (kNcodeIn1 + q - 1), in2 = 1u << (kNcodeIn2 + q - 1);
        if ((code & miss) && !(code & in1)) mom = true;
        int32_t dummy;
        if (lab_at(dom, i - vx, j - vy, nx, ny, bc_y, pitch, &dummy)) {
            const int xi = i - vx < 0 ? i - vx + nx : (i - vx >= nx ? i - vx - nx : i - vx);
            const int xj = (j - vy + ny) % ny;
            const uint32_t c1 = ncode_links(dom, xi, xj, nx, ny, bc_y, pitch);
            if ((c1 & miss) && (c1 & in1)) mom = true;
        }
        if (lab_at(dom, i - 2 * vx, j - 2 * vy, nx, ny, bc_y, pitch, &dummy)) {
            const int xi = ((i - 2 * vx) % nx + nx) % nx;
            const int xj = ((j - 2 * vy) % ny + ny) % ny;
            const uint32_t c2 = ncode_links(dom, xi, xj, nx, ny, bc_y, pitch);
            if ((c2 & miss) && (c2 & in2)) mom = true;
        }
    }
    if (mom) code |= 1u << kNcodeMom;
    ncode[(int64_t)j * pitch + i] = (uint16_t)code;
}

cudaError_t launch_make_ncode(const int32_t* dom, uint16_t* ncode, int nx, int ny, int bc_y,
                              int64_t pitch, cudaStream_t s) {
    make_ncode_kernel<<<dim3((nx + 127) / 128, ny), 128, 0, s>>>(dom, ncode, nx, ny, bc_y, pitch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Species moments of stored populations at the same node (no streaming):
// phi, jx, jy per species in the compute type, the moments a run starts from.
template <typename T, typename C>
__global__ void species_moments_kernel(int S, int nx, int ny, int64_t pitch, int64_t plane,
                                       const T* g, C* mom, Coefs<C> k, bool scaled) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= nx || j >= ny) return;
    const int64_t node = (int64_t)j * pitch + i;
    const uint64_t pol = l2_evict_normal();
    for (int s = 0; s < S; ++s) {
        C v[5];
        for (int q = 0; q < 5; ++q) {
            v[q] = Store<T, C>::ld(g + (int64_t)(5 * s + q) * plane + node, pol);
            if (scaled) v[q] *= k.gscale[q];
        }
        C* M = mom + (int64_t)3 * s * plane;
        M[node] = v[0] + v[1] + v[2] + v[3] + v[4];
        M[plane + node] = v[1] - v[3];
        M[2 * plane + node] = v[2] - v[4];
    }
}

cudaError_t launch_species_moments(int precision, int n_species, int nx, int ny, int64_t pitch,
                                   int64_t plane, const void* g, void* mom, const void* coefs,
                                   cudaStream_t s) {
    if (n_species <= 0) return cudaSuccess;
    const dim3 grid((nx + 127) / 128, ny), block(128);
    if (precision == LBIB_FP64)
        species_moments_kernel<double, double><<<grid, block, 0, s>>>(
            n_species, nx, ny, pitch, plane, static_cast<const double*>(g),
            static_cast<double*>(mom), *static_cast<const Coefs<double>*>(coefs), false);
    else if (precision == LBIB_FP32)
        species_moments_kernel<float, float><<<grid, block, 0, s>>>(
            n_species, nx, ny, pitch, plane, static_cast<const float*>(g),
            static_cast<float*>(mom), *static_cast<const Coefs<float>*>(coefs), false);
    else
        species_moments_kernel<__half, float><<<grid, block, 0, s>>>(
            n_species, nx, ny, pitch, plane, static_cast<const __half*>(g),
            static_cast<float*>(mom), *static_cast<const Coefs<float>*>(coefs), true);
    return cudaGetLastError();
}

}  // namespace lbib
