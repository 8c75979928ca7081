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

#include "lattice_kernel.cuh"

namespace lbib {

// ---------------------------------------------------------------------------
// FP16 storage, two nodes per thread.  One population of a node is two
// bytes, so a thread that reads one node keeps few bytes in flight; here a
// thread owns the pair (x0, x0 + 1), x0 = 2 * (thread index in x), and every
// population moves as one 32-bit word of two halves (rows start 64-aligned,
// so a warp covers 64 consecutive nodes of one row).  A direction with an
// x-component pulls the pair shifted by one node: its two halves are the
// neighbouring halves of the thread's own aligned word and of the adjacent
// lane's (a warp shuffle); the first and the last lane of a warp, and the
// last pair of a row, load the word beyond the warp themselves (periodic in
// x).  Both nodes collide at once in packed FP32 arithmetic (collide_node
// on float2), per node the same operations as the one-node update.
// Register budget of the pair kernel (CTAs of 128 threads per SM; the packed
// values of two nodes take register pairs): 64 without species, 72 with one,
// 102 with two, 128 with three or four (no spills).
template <int S>
struct PairOccupancy {
    static constexpr int kMinBlocks = S == 0 ? 8 : (S == 1 ? 7 : (S == 2 ? 6 : 4));
};

__device__ __forceinline__ uint32_t ldw(const uint32_t* p, uint64_t pol) {
    return ld_stream(p, pol);
}

// the pair (x0 - 1, x0) from the aligned word a = (x0, x0 + 1) and e, the
// word (x0 - 2, x0 - 1) loaded by the lanes with own_l set
__device__ __forceinline__ uint32_t pair_from_left(uint32_t a, uint32_t e, bool own_l) {
    const uint32_t up = __shfl_up_sync(0xffffffffu, a, 1);
    return __funnelshift_r(own_l ? e : up, a, 16);
}
// the pair (x0 + 1, x0 + 2) from a and e, the word (x0 + 2, x0 + 3) loaded by
// the lanes with own_r set
__device__ __forceinline__ uint32_t pair_from_right(uint32_t a, uint32_t e, bool own_r) {
    const uint32_t dn = __shfl_down_sync(0xffffffffu, a, 1);
    return __funnelshift_r(a, own_r ? e : dn, 16);
}

__device__ __forceinline__ uint32_t pack_halves(float2 v) {
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <int S, bool WALLS, int FORCING>
__global__ void __launch_bounds__(kLatticeThreads, PairOccupancy<S>::kMinBlocks)
    lattice_pair_kernel(LatticeArgs a, Coefs<float> k) {
    using C = float;
    constexpr int SS = S > 0 ? S : 1;
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    // whole warps past the row end leave; the others keep every lane for the
    // shuffles (lanes past the end load and store nothing)
    if (2 * (t - lane) >= a.nx || y >= a.ny) return;
    const int x0 = 2 * t;
    bool valid = x0 < a.nx;
    const bool lo_wall = WALLS && (y == 0);
    const bool hi_wall = WALLS && (y == a.ny - 1);
    const int ym = (y == 0) ? a.ny - 1 : y - 1;
    const int yp = (y == a.ny - 1) ? 0 : y + 1;
    const int64_t P2 = a.plane >> 1;  // words per plane
    // in-plane indices are 32-bit (a plane holds fewer than 2^31 nodes); the
    // plane bases (F + q * P2 and so on) are the same for every thread
    const int r0 = y * (int)a.pitch;
    const int rm = ym * (int)a.pitch;
    const int rp = yp * (int)a.pitch;
    const int node = r0 + x0;
    const int w = node >> 1, wm = (rm + x0) >> 1, wp = (rp + x0) >> 1;
    const int xl = (x0 == 0) ? a.nx - 2 : x0 - 2;
    const int xr = (x0 + 2 >= a.nx) ? 0 : x0 + 2;
    const bool own_l = valid && lane == 0;
    const bool own_r = valid && (lane == 31 || x0 + 2 >= a.nx);
    const int l0 = (r0 + xl) >> 1, lm = (rm + xl) >> 1, lp = (rp + xl) >> 1;
    const int q0 = (r0 + xr) >> 1, qm = (rm + xr) >> 1, qp = (rp + xr) >> 1;
    // the checking build: the word indices inside the plane, the 16-byte
    // accesses of the pair aligned; a lane that fails loads and stores
    // nothing but still takes part in the warp's shuffles
    if (valid &&
        (!LBIB_CHK_INDEX(a.diag, kSitePairIndex,
                         (int64_t)max(max(max(wm, wp), max(lm, lp)), max(max(qm, qp), w)), P2) ||
         !LBIB_CHK_ACCESS(a.diag, kSitePairAlign, static_cast<const float4*>(a.u) + (node >> 1),
                          16, nullptr, nullptr) ||
         !LBIB_CHK_ACCESS(a.diag, kSitePairAlign, static_cast<const float4*>(a.force) + (node >> 1),
                          16, nullptr, nullptr) ||
         !LBIB_CHK_INDEX(a.diag, kSiteMask, (int64_t)(node >> 7), mask_words(a.plane))))
        valid = false;

    // ---- every population word first (written two launches back: L2 path)
    const uint64_t pol = a.l2_first ? l2_evict_first() : l2_evict_normal();
    const uint32_t* F = static_cast<const uint32_t*>(a.fsrc);
    uint32_t r[9], e[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) r[q] = e[q] = 0u;
    if (valid) {
        r[0] = ldw(F + w, pol);
        r[1] = ldw((F + 1 * P2) + w, pol);
        r[3] = ldw((F + 3 * P2) + w, pol);
        r[2] = lo_wall ? ldw((F + 4 * P2) + w, pol) : ldw((F + 2 * P2) + wm, pol);
        r[4] = hi_wall ? ldw((F + 2 * P2) + w, pol) : ldw((F + 4 * P2) + wp, pol);
        if (lo_wall) {  // half-way bounce-back at y = -1/2
            r[5] = ldw((F + 7 * P2) + w, pol);
            r[6] = ldw((F + 8 * P2) + w, pol);
        } else {
            r[5] = ldw((F + 5 * P2) + wm, pol);
            r[6] = ldw((F + 6 * P2) + wm, pol);
        }
        if (hi_wall) {  // at y = ny - 1/2
            r[7] = ldw((F + 5 * P2) + w, pol);
            r[8] = ldw((F + 6 * P2) + w, pol);
        } else {
            r[7] = ldw((F + 7 * P2) + wp, pol);
            r[8] = ldw((F + 8 * P2) + wp, pol);
        }
        if (own_l) {
            e[1] = ldw((F + 1 * P2) + l0, pol);
            if (!lo_wall) e[5] = ldw((F + 5 * P2) + lm, pol);
            if (!hi_wall) e[8] = ldw((F + 8 * P2) + lp, pol);
        }
        if (own_r) {
            e[3] = ldw((F + 3 * P2) + q0, pol);
            if (!lo_wall) e[6] = ldw((F + 6 * P2) + qm, pol);
            if (!hi_wall) e[7] = ldw((F + 7 * P2) + qp, pol);
        }
    }
    uint32_t rg[SS][5], eg[SS][2];
#pragma unroll
    for (int s = 0; s < SS; ++s) {
        rg[s][0] = rg[s][1] = rg[s][2] = rg[s][3] = rg[s][4] = 0u;
        eg[s][0] = eg[s][1] = 0u;
    }
    if (valid) {
        const uint32_t* Gi = static_cast<const uint32_t*>(a.gsrc);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint32_t* B = Gi + (int64_t)s * 5 * P2;
            rg[s][0] = ldw(B + w, pol);
            rg[s][1] = ldw((B + 1 * P2) + w, pol);
            rg[s][3] = ldw((B + 3 * P2) + w, pol);
            rg[s][2] = lo_wall ? ldw((B + 4 * P2) + w, pol) : ldw((B + 2 * P2) + wm, pol);
            rg[s][4] = hi_wall ? ldw((B + 2 * P2) + w, pol) : ldw((B + 4 * P2) + wp, pol);
            if (own_l) eg[s][0] = ldw((B + 1 * P2) + l0, pol);
            if (own_r) eg[s][1] = ldw((B + 3 * P2) + q0, pol);
        }
    }
    // the IB kernel launched just before wrote the force, label and mask
    // planes: wait for it, then let the next IB launch start
    griddep_wait();
    griddep_launch_dependents();

    // the shifted pairs (every lane takes part in the shuffles)
    r[1] = pair_from_left(r[1], e[1], own_l);
    r[3] = pair_from_right(r[3], e[3], own_r);
    {
        const uint32_t p5 = pair_from_left(r[5], e[5], own_l);
        const uint32_t p6 = pair_from_right(r[6], e[6], own_r);
        const uint32_t p7 = pair_from_right(r[7], e[7], own_r);
        const uint32_t p8 = pair_from_left(r[8], e[8], own_l);
        if (!lo_wall) {
            r[5] = p5;
            r[6] = p6;
        }
        if (!hi_wall) {
            r[7] = p7;
            r[8] = p8;
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        rg[s][1] = pair_from_left(rg[s][1], eg[s][0], own_l);
        rg[s][3] = pair_from_right(rg[s][3], eg[s][1], own_r);
    }
    if (!valid) return;

    // spread force, labels and source bits of the pair's 4-node group
    float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
    uint2 label = make_uint2(kOutside, kOutside);
    uint32_t sb2 = 0u;
    bool fhit = false, lhit = false, shit = false;
    uint32_t clear = 0u;  // lane 0: which masks hold bits of the warp's 16 groups
    const int grp = node >> 2;
    if (a.ib) {
        if (a.fmask) {
            const int sh = (int)(grp & 31);
            const uint32_t fw = a.fmask[grp >> 5] >> sh;
            const uint32_t lw = a.lmask[grp >> 5] >> sh;
            const uint32_t sw = a.smask[grp >> 5] >> sh;
            fhit = fw & 1u;
            lhit = lw & 1u;
            shit = sw & 1u;
            clear = ((fw & 0xFFFFu) ? 1u : 0u) | ((lw & 0xFFFFu) ? 2u : 0u) |
                    ((sw & 0xFFFFu) ? 4u : 0u);
        } else {
            fhit = shit = true;
            lhit = a.id != nullptr;
        }
        if (fhit) fv = static_cast<const float4*>(a.force)[node >> 1];
        if (lhit) label = reinterpret_cast<const uint2*>(a.id)[node >> 1];
        if (shit) sb2 = reinterpret_cast<const unsigned short*>(a.src)[node >> 1];
    }

    // ---- the collision of both nodes at once (packed FP32: x = node x0,
    // y = node x0 + 1)
    float2 d[9], g[SS][5], ph[SS], rho, ux, uy;
#pragma unroll
    for (int q = 0; q < 9; ++q) d[q] = __half22float2(*reinterpret_cast<const __half2*>(&r[q]));
#pragma unroll
    for (int s = 0; s < SS; ++s)
#pragma unroll
        for (int q = 0; q < 5; ++q)
            g[s][q] = __half22float2(*reinterpret_cast<const __half2*>(&rg[s][q]));
    collide_node<float2, S, FORCING, true>(k, d, g, make_float2(fv.x, fv.z),
                                           make_float2(fv.y, fv.w), sb2 & 0xFFu, sb2 >> 8, rho,
                                           ux, uy, ph);

    uint32_t* G = static_cast<uint32_t*>(a.fdst);
#pragma unroll
    for (int q = 0; q < 9; ++q) (G + q * P2)[w] = pack_halves(d[q]);
    if (S > 0) {
        uint32_t* Go = static_cast<uint32_t*>(a.gdst);
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int q = 0; q < 5; ++q) (Go + (int64_t)(s * 5 + q) * P2)[w] = pack_halves(g[s][q]);
            if (a.out)
                reinterpret_cast<float2*>(static_cast<C*>(a.phi) + (int64_t)s * a.plane)[node >> 1] =
                    ph[s];
        }
    }

    // velocity where the interpolation will read it, resets, outputs, masks
    if (a.out || fhit)
        st_keep(static_cast<float4*>(a.u) + (node >> 1), make_float4(ux.x, uy.x, ux.y, uy.y));
    if (a.ib) {
        if (fhit) st_keep(static_cast<float4*>(a.force) + (node >> 1), make_float4(0.f, 0.f, 0.f, 0.f));
        if (lhit) reinterpret_cast<uint2*>(a.id)[node >> 1] = make_uint2(kOutside, kOutside);
        if (shit) reinterpret_cast<unsigned short*>(a.src)[node >> 1] = 0;
        if (a.out) {
            reinterpret_cast<uint2*>(a.id_out)[node >> 1] = label;
            static_cast<float4*>(a.force_out)[node >> 1] = fv;
        }
        // lane 0 clears the warp's 16 group bits (64 nodes of one row, 64-aligned)
        if (clear && lane == 0) {
            const int sh = (int)(grp & 31);
            if (clear & 1u) atomicAnd(a.fmask + (grp >> 5), ~(0xFFFFu << sh));
            if (clear & 2u) atomicAnd(a.lmask + (grp >> 5), ~(0xFFFFu << sh));
            if (clear & 4u) atomicAnd(a.smask + (grp >> 5), ~(0xFFFFu << sh));
        }
    }
    if (a.out) reinterpret_cast<float2*>(a.rho)[node >> 1] = rho;
    if (!(rho.x > 0.f) || !isfinite(ux.x) || !isfinite(uy.x) || !(rho.y > 0.f) ||
        !isfinite(ux.y) || !isfinite(uy.y))
        atomicOr(a.diag + kDiagNonFinite, 1u);
}

template <typename T, typename C, int S, bool WALLS, int FORCING>
static cudaError_t launch3(const LatticeArgs& a, const void* coefs, dim3 block, cudaStream_t s,
                           bool pdl, bool pairs) {
    // the group masks are cleared per warp: a warp must be 32 nodes of one row
    if (a.fmask && block.x % 32 != 0) return cudaErrorInvalidConfiguration;
    if (block.x * block.y * block.z > (unsigned)kLatticeThreads) return cudaErrorInvalidConfiguration;
    dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
    const Coefs<C>& k = *static_cast<const Coefs<C>*>(coefs);
    constexpr bool SC = std::is_same<T, __half>::value;
    if constexpr (SC) {
        // two nodes per thread when the rows hold whole pairs
        // (confined species read their neighbours' domains, mass sources and
        // pressure nodes are per node: one node per thread)
        if (pairs && !a.dom && !a.msrc && !a.pnode && !a.nsrc && a.nx % 2 == 0 && a.pitch % 64 == 0 && a.plane % 2 == 0) {
            const dim3 pb(kLatticeThreads, 1, 1);
            const dim3 pg((a.nx / 2 + kLatticeThreads - 1) / kLatticeThreads, a.ny);
            return launch_kernel(lattice_pair_kernel<S, WALLS, FORCING>, pg, pb, 0, s, pdl, a,
                                 k);
        }
    }
    return launch_kernel(lattice_kernel<T, C, S, WALLS, FORCING, SC, false>, grid, block, 0, s,
                         pdl, a, k);
}

template <typename T, typename C, int S>
static cudaError_t launch2(int bc_y, int forcing, const LatticeArgs& a, const void* coefs,
                           dim3 block, cudaStream_t s, bool pdl, bool pairs) {
    if (bc_y) {
        return forcing ? launch3<T, C, S, true, 1>(a, coefs, block, s, pdl, pairs)
                       : launch3<T, C, S, true, 0>(a, coefs, block, s, pdl, pairs);
    }
    return forcing ? launch3<T, C, S, false, 1>(a, coefs, block, s, pdl, pairs)
                   : launch3<T, C, S, false, 0>(a, coefs, block, s, pdl, pairs);
}

template <typename T, typename C>
static cudaError_t launch1(int n_species, int bc_y, int forcing, const LatticeArgs& a,
                           const void* coefs, dim3 block, cudaStream_t s, bool pdl, bool pairs) {
    switch (n_species) {
        case 0: return launch2<T, C, 0>(bc_y, forcing, a, coefs, block, s, pdl, pairs);
        case 1: return launch2<T, C, 1>(bc_y, forcing, a, coefs, block, s, pdl, pairs);
        case 2: return launch2<T, C, 2>(bc_y, forcing, a, coefs, block, s, pdl, pairs);
        case 3: return launch2<T, C, 3>(bc_y, forcing, a, coefs, block, s, pdl, pairs);
        default: return launch2<T, C, 4>(bc_y, forcing, a, coefs, block, s, pdl, pairs);
    }
}

bool lattice_l2_first(int precision, int n_species, int64_t plane) {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int es = precision == LBIB_FP64 ? 8 : (precision == LBIB_FP32 ? 4 : 2);
    const double bytes = 2.0 * (9 + 5 * n_species) * (double)plane * es;
    return bytes <= 1.5 * (double)l2;
}

cudaError_t launch_lattice(int precision, int n_species, int bc_y, int forcing,
                           const LatticeArgs& a, const void* coefs, dim3 block, cudaStream_t s,
                           bool pdl, bool pairs) {
    // confined species: the kernels with their paths compiled in
    if (a.dom && n_species > 0)
        return launch_lattice_confined(precision, n_species, bc_y, forcing, a, coefs, block, s,
                                       pdl);
    if (precision == LBIB_FP64)
        return launch1<double, double>(n_species, bc_y, forcing, a, coefs, block, s, pdl, pairs);
    if (precision == LBIB_FP32)
        return launch1<float, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl, pairs);
    return launch1<__half, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl, pairs);
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
        C gq = k.w5c[q == 0 ? 0 : 1] * C(v);
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
