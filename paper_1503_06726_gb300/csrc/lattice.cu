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

// ---------------------------------------------------------------------------
// FP16 storage, four nodes per thread.  The pair update's per-thread work
// that does not grow with the nodes (indices, group-mask reads, the shuffles
// of the x-shifted words, the edge loads, the non-finite test) is shared by
// four nodes here: a thread owns the quad (x0 .. x0 + 3), x0 = 4 * (thread
// index in x), and every population moves as one 64-bit word of four halves
// (rows start 64-aligned, so a warp covers 128 consecutive nodes of one
// row).  A direction with an x-component pulls the quad shifted by one node:
// its halves are three of the thread's own word and one of the adjacent
// lane's (a warp shuffle of the 32-bit half that holds it); the first and the
// last lane of a warp, and the last quad of a row, load that 32-bit word
// themselves (periodic in x).  The quad is two pairs, each collided in packed
// FP32 arithmetic (collide_node on float2): per node the same operations as
// the one-node update.  A quad is exactly one 4-node group of the masks.
// Register budget (CTAs of 128 threads per SM): 128 registers with at most
// one species, 168 with two, 255 with more.
template <int S>
struct QuadOccupancy {
    static constexpr int kMinBlocks = S <= 1 ? 4 : (S == 2 ? 3 : 2);
};

__device__ __forceinline__ uint2 ldw2(const uint2* p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.cg.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
    return v;
}

// the quad (x0 - 1 .. x0 + 2) from a = (x0 .. x0 + 3) and e, the 32-bit word
// (x0 - 2, x0 - 1) loaded by the lanes with own_l set
__device__ __forceinline__ uint2 quad_from_left(uint2 a, uint32_t e, bool own_l) {
    const uint32_t up = __shfl_up_sync(0xffffffffu, a.y, 1);
    const uint32_t lw = own_l ? e : up;
    return make_uint2(__funnelshift_l(lw, a.x, 16), __funnelshift_l(a.x, a.y, 16));
}
// the quad (x0 + 1 .. x0 + 4) from a and e, the 32-bit word (x0 + 4, x0 + 5)
// loaded by the lanes with own_r set
__device__ __forceinline__ uint2 quad_from_right(uint2 a, uint32_t e, bool own_r) {
    const uint32_t dn = __shfl_down_sync(0xffffffffu, a.x, 1);
    const uint32_t rw = own_r ? e : dn;
    return make_uint2(__funnelshift_r(a.x, a.y, 16), __funnelshift_r(a.y, rw, 16));
}

__device__ __forceinline__ float2 lo_pair(uint2 v) {
    return __half22float2(*reinterpret_cast<const __half2*>(&v.x));
}
__device__ __forceinline__ float2 hi_pair(uint2 v) {
    return __half22float2(*reinterpret_cast<const __half2*>(&v.y));
}

// The update of one quad after its population words are in registers (r,
// rg: the shifted words assembled): the IB planes of its group, the
// collision of its two pairs, the stores.  fmw, lmw, smw: the group's force,
// label and source mask words, read when the masks are in use.
template <int S, int FORCING>
__device__ __forceinline__ void quad_update(const LatticeArgs& a, const Coefs<float>& k,
                                            int node, int lane, const uint2 (&r)[9],
                                            const uint2 (&rg)[S > 0 ? S : 1][5],
                                            const uint32_t* fmw, const uint32_t* lmw,
                                            const uint32_t* smw) {
    using C = float;
    constexpr int SS = S > 0 ? S : 1;
    const int64_t P4 = a.plane >> 2;
    const int w = node >> 2;
    // spread force, labels and source bits of the quad (one 4-node group)
    float4 fv0 = make_float4(0.f, 0.f, 0.f, 0.f), fv1 = fv0;
    uint4 label = make_uint4(kOutside, kOutside, kOutside, kOutside);
    uint32_t sb4 = 0u;
    bool fhit = false, lhit = false, shit = false;
    // the lanes that clear mask bits: lane 0, and a lane whose group opens a
    // mask word inside the warp (rows that start at an odd multiple of 64
    // nodes); each clears its bits up to the warp's or the word's end
    uint32_t clear = 0u, seg = 0u;
    const int grp = node >> 2;
    if (a.ib) {
        if (a.fmask) {
            const int sh = (int)(grp & 31);
            const uint32_t fw = *fmw;
            const uint32_t lw = *lmw;
            const uint32_t sw = *smw;
            fhit = (fw >> sh) & 1u;
            lhit = (lw >> sh) & 1u;
            shit = (sw >> sh) & 1u;
            if (lane == 0 || sh == 0) {
                const int n = min(32 - sh, 32 - lane);
                seg = (n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u)) << sh;
                clear = ((fw & seg) ? 1u : 0u) | ((lw & seg) ? 2u : 0u) | ((sw & seg) ? 4u : 0u);
            }
        } else {
            fhit = shit = true;
            lhit = a.id != nullptr;
        }
        if (fhit) {
            fv0 = static_cast<const float4*>(a.force)[node >> 1];
            fv1 = static_cast<const float4*>(a.force)[(node >> 1) + 1];
        }
        if (lhit) label = reinterpret_cast<const uint4*>(a.id)[node >> 2];
        if (shit) sb4 = reinterpret_cast<const uint32_t*>(a.src)[node >> 2];
    }

    // ---- the collision of the two pairs (packed FP32: A = nodes x0, x0 + 1;
    // B = nodes x0 + 2, x0 + 3)
    float2 dA[9], dB[9], gA[SS][5], gB[SS][5], phA[SS], phB[SS];
    float2 rhoA, rhoB, uxA, uxB, uyA, uyB;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        dA[q] = lo_pair(r[q]);
        dB[q] = hi_pair(r[q]);
    }
#pragma unroll
    for (int s = 0; s < SS; ++s)
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            gA[s][q] = lo_pair(rg[s][q]);
            gB[s][q] = hi_pair(rg[s][q]);
        }
    collide_node<float2, S, FORCING, true>(k, dA, gA, make_float2(fv0.x, fv0.z),
                                           make_float2(fv0.y, fv0.w), sb4 & 0xFFu,
                                           (sb4 >> 8) & 0xFFu, rhoA, uxA, uyA, phA);
    collide_node<float2, S, FORCING, true>(k, dB, gB, make_float2(fv1.x, fv1.z),
                                           make_float2(fv1.y, fv1.w), (sb4 >> 16) & 0xFFu,
                                           sb4 >> 24, rhoB, uxB, uyB, phB);

    uint2* G = static_cast<uint2*>(a.fdst);
#pragma unroll
    for (int q = 0; q < 9; ++q) (G + q * P4)[w] = make_uint2(pack_halves(dA[q]), pack_halves(dB[q]));
    if (S > 0) {
        uint2* Go = static_cast<uint2*>(a.gdst);
#pragma unroll
        for (int s = 0; s < S; ++s) {
#pragma unroll
            for (int q = 0; q < 5; ++q)
                (Go + (int64_t)(s * 5 + q) * P4)[w] =
                    make_uint2(pack_halves(gA[s][q]), pack_halves(gB[s][q]));
            if (a.out)
                reinterpret_cast<float4*>(static_cast<C*>(a.phi) + (int64_t)s * a.plane)[node >> 2] =
                    make_float4(phA[s].x, phA[s].y, phB[s].x, phB[s].y);
        }
    }

    // velocity where the interpolation will read it, resets, outputs, masks
    if (a.out || fhit) {
        float4* U = static_cast<float4*>(a.u) + (node >> 1);
        st_keep(U, make_float4(uxA.x, uyA.x, uxA.y, uyA.y));
        st_keep(U + 1, make_float4(uxB.x, uyB.x, uxB.y, uyB.y));
    }
    if (a.ib) {
        if (fhit) {
            float4* Fo = static_cast<float4*>(a.force) + (node >> 1);
            st_keep(Fo, make_float4(0.f, 0.f, 0.f, 0.f));
            st_keep(Fo + 1, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        if (lhit)
            reinterpret_cast<uint4*>(a.id)[node >> 2] =
                make_uint4(kOutside, kOutside, kOutside, kOutside);
        if (shit) reinterpret_cast<uint32_t*>(a.src)[node >> 2] = 0u;
        if (a.out) {
            reinterpret_cast<uint4*>(a.id_out)[node >> 2] = label;
            static_cast<float4*>(a.force_out)[node >> 1] = fv0;
            static_cast<float4*>(a.force_out)[(node >> 1) + 1] = fv1;
        }
        if (clear) {
            if (clear & 1u) atomicAnd(a.fmask + (grp >> 5), ~seg);
            if (clear & 2u) atomicAnd(a.lmask + (grp >> 5), ~seg);
            if (clear & 4u) atomicAnd(a.smask + (grp >> 5), ~seg);
        }
    }
    if (a.out)
        reinterpret_cast<float4*>(a.rho)[node >> 2] = make_float4(rhoA.x, rhoA.y, rhoB.x, rhoB.y);
    const bool bad = !(rhoA.x > 0.f) || !(rhoA.y > 0.f) || !(rhoB.x > 0.f) || !(rhoB.y > 0.f) ||
                     !isfinite(uxA.x) || !isfinite(uyA.x) || !isfinite(uxA.y) ||
                     !isfinite(uyA.y) || !isfinite(uxB.x) || !isfinite(uyB.x) ||
                     !isfinite(uxB.y) || !isfinite(uyB.y);
    if (bad) atomicOr(a.diag + kDiagNonFinite, 1u);
}

template <int S, bool WALLS, int FORCING>
__global__ void __launch_bounds__(kLatticeThreads, QuadOccupancy<S>::kMinBlocks)
    lattice_quad_kernel(LatticeArgs a, Coefs<float> k) {
    using C = float;
    constexpr int SS = S > 0 ? S : 1;
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    // whole warps past the row end leave; the others keep every lane for the
    // shuffles (lanes past the end load and store nothing)
    if (4 * (t - lane) >= a.nx || y >= a.ny) return;
    const int x0 = 4 * t;
    bool valid = x0 < a.nx;
    const bool lo_wall = WALLS && (y == 0);
    const bool hi_wall = WALLS && (y == a.ny - 1);
    const int ym = (y == 0) ? a.ny - 1 : y - 1;
    const int yp = (y == a.ny - 1) ? 0 : y + 1;
    const int64_t P4 = a.plane >> 2;  // 64-bit words per plane
    const int64_t P2 = a.plane >> 1;  // 32-bit words per plane (the edge words)
    // in-plane indices are 32-bit (a plane holds fewer than 2^31 nodes)
    const int r0 = y * (int)a.pitch;
    const int rm = ym * (int)a.pitch;
    const int rp = yp * (int)a.pitch;
    const int node = r0 + x0;
    const int w = node >> 2, wm = (rm + x0) >> 2, wp = (rp + x0) >> 2;
    const int xl = (x0 == 0) ? a.nx - 2 : x0 - 2;
    const int xr = (x0 + 4 >= a.nx) ? 0 : x0 + 4;
    const bool own_l = valid && lane == 0;
    const bool own_r = valid && (lane == 31 || x0 + 4 >= a.nx);
    const int l0 = (r0 + xl) >> 1, lm = (rm + xl) >> 1, lp = (rp + xl) >> 1;
    const int q0 = (r0 + xr) >> 1, qm = (rm + xr) >> 1, qp = (rp + xr) >> 1;
    // the checking build: the word indices inside the plane, the 16-byte
    // accesses of the quad aligned; a lane that fails loads and stores
    // nothing but still takes part in the warp's shuffles
    if (valid &&
        (!LBIB_CHK_INDEX(a.diag, kSitePairIndex, (int64_t)max(max(wm, wp), w), P4) ||
         !LBIB_CHK_INDEX(a.diag, kSitePairIndex,
                         (int64_t)max(max(max(lm, lp), max(qm, qp)), max(l0, q0)), P2) ||
         !LBIB_CHK_ACCESS(a.diag, kSitePairAlign, static_cast<const float4*>(a.u) + (node >> 1),
                          16, nullptr, nullptr) ||
         !LBIB_CHK_ACCESS(a.diag, kSitePairAlign, static_cast<const float4*>(a.force) + (node >> 1),
                          16, nullptr, nullptr) ||
         !LBIB_CHK_INDEX(a.diag, kSiteMask, (int64_t)(node >> 7), mask_words(a.plane))))
        valid = false;

    // ---- every population word first (written two launches back: L2 path)
    const uint64_t pol = a.l2_first ? l2_evict_first() : l2_evict_normal();
    const uint2* F = static_cast<const uint2*>(a.fsrc);
    const uint32_t* F1 = static_cast<const uint32_t*>(a.fsrc);
    uint2 r[9];
    uint32_t e[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        r[q] = make_uint2(0u, 0u);
        e[q] = 0u;
    }
    if (valid) {
        r[0] = ldw2(F + w, pol);
        r[1] = ldw2((F + 1 * P4) + w, pol);
        r[3] = ldw2((F + 3 * P4) + w, pol);
        r[2] = lo_wall ? ldw2((F + 4 * P4) + w, pol) : ldw2((F + 2 * P4) + wm, pol);
        r[4] = hi_wall ? ldw2((F + 2 * P4) + w, pol) : ldw2((F + 4 * P4) + wp, pol);
        if (lo_wall) {  // half-way bounce-back at y = -1/2
            r[5] = ldw2((F + 7 * P4) + w, pol);
            r[6] = ldw2((F + 8 * P4) + w, pol);
        } else {
            r[5] = ldw2((F + 5 * P4) + wm, pol);
            r[6] = ldw2((F + 6 * P4) + wm, pol);
        }
        if (hi_wall) {  // at y = ny - 1/2
            r[7] = ldw2((F + 5 * P4) + w, pol);
            r[8] = ldw2((F + 6 * P4) + w, pol);
        } else {
            r[7] = ldw2((F + 7 * P4) + wp, pol);
            r[8] = ldw2((F + 8 * P4) + wp, pol);
        }
        if (own_l) {
            e[1] = ldw((F1 + 1 * P2) + l0, pol);
            if (!lo_wall) e[5] = ldw((F1 + 5 * P2) + lm, pol);
            if (!hi_wall) e[8] = ldw((F1 + 8 * P2) + lp, pol);
        }
        if (own_r) {
            e[3] = ldw((F1 + 3 * P2) + q0, pol);
            if (!lo_wall) e[6] = ldw((F1 + 6 * P2) + qm, pol);
            if (!hi_wall) e[7] = ldw((F1 + 7 * P2) + qp, pol);
        }
    }
    uint2 rg[SS][5];
    uint32_t eg[SS][2];
#pragma unroll
    for (int s = 0; s < SS; ++s) {
#pragma unroll
        for (int q = 0; q < 5; ++q) rg[s][q] = make_uint2(0u, 0u);
        eg[s][0] = eg[s][1] = 0u;
    }
    if (valid) {
        const uint2* Gi = static_cast<const uint2*>(a.gsrc);
        const uint32_t* Gi1 = static_cast<const uint32_t*>(a.gsrc);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const uint2* B = Gi + (int64_t)s * 5 * P4;
            const uint32_t* B1 = Gi1 + (int64_t)s * 5 * P2;
            rg[s][0] = ldw2(B + w, pol);
            rg[s][1] = ldw2((B + 1 * P4) + w, pol);
            rg[s][3] = ldw2((B + 3 * P4) + w, pol);
            rg[s][2] = lo_wall ? ldw2((B + 4 * P4) + w, pol) : ldw2((B + 2 * P4) + wm, pol);
            rg[s][4] = hi_wall ? ldw2((B + 2 * P4) + w, pol) : ldw2((B + 4 * P4) + wp, pol);
            if (own_l) eg[s][0] = ldw((B1 + 1 * P2) + l0, pol);
            if (own_r) eg[s][1] = ldw((B1 + 3 * P2) + q0, pol);
        }
    }
    // the IB kernel launched just before wrote the force, label and mask
    // planes: wait for it, then let the next IB launch start
    griddep_wait();
    griddep_launch_dependents();

    // the shifted quads (every lane takes part in the shuffles)
    r[1] = quad_from_left(r[1], e[1], own_l);
    r[3] = quad_from_right(r[3], e[3], own_r);
    {
        const uint2 p5 = quad_from_left(r[5], e[5], own_l);
        const uint2 p6 = quad_from_right(r[6], e[6], own_r);
        const uint2 p7 = quad_from_right(r[7], e[7], own_r);
        const uint2 p8 = quad_from_left(r[8], e[8], own_l);
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
        rg[s][1] = quad_from_left(rg[s][1], eg[s][0], own_l);
        rg[s][3] = quad_from_right(rg[s][3], eg[s][1], own_r);
    }
    if (!valid) return;

    const int mword = node >> 7;  // the group's mask word
    const bool m = a.fmask != nullptr;
    quad_update<S, FORCING>(a, k, node, lane, r, rg, m ? a.fmask + mword : nullptr,
                            m ? a.lmask + mword : nullptr, m ? a.smask + mword : nullptr);
}

template <typename T, typename C, int S, bool WALLS, int FORCING>
static cudaError_t launch3(const LatticeArgs& a, const void* coefs, dim3 block, cudaStream_t s,
                           bool pdl, int npt) {
    // the group masks are cleared per warp: a warp must be 32 nodes of one row
    if (a.fmask && block.x % 32 != 0) return cudaErrorInvalidConfiguration;
    if (block.x * block.y * block.z > (unsigned)kLatticeThreads) return cudaErrorInvalidConfiguration;
    dim3 grid((a.nx + block.x - 1) / block.x, (a.ny + block.y - 1) / block.y);
    const Coefs<C>& k = *static_cast<const Coefs<C>*>(coefs);
    constexpr bool SC = std::is_same<T, __half>::value;
    if constexpr (SC) {
        // by default two nodes per thread (the pair update)
        if (npt == 0) npt = 2;
        // two or four nodes per thread when the rows hold whole pairs or
        // quads (confined species read their neighbours' domains, mass
        // sources and pressure nodes are per node: one node per thread)
        const bool plain = !a.dom && !a.msrc && !a.pnode && !a.nsrc && a.pitch % 64 == 0;
        if (npt == 4 && plain && a.nx % 4 == 0 && a.plane % 4 == 0) {
            const dim3 qb(kLatticeThreads, 1, 1);
            const dim3 qg((a.nx / 4 + kLatticeThreads - 1) / kLatticeThreads, a.ny);
            return launch_kernel(lattice_quad_kernel<S, WALLS, FORCING>, qg, qb, 0, s, pdl, a,
                                 k);
        }
        if (npt >= 2 && plain && a.nx % 2 == 0 && a.plane % 2 == 0) {
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
                           dim3 block, cudaStream_t s, bool pdl, int npt) {
    if (bc_y) {
        return forcing ? launch3<T, C, S, true, 1>(a, coefs, block, s, pdl, npt)
                       : launch3<T, C, S, true, 0>(a, coefs, block, s, pdl, npt);
    }
    return forcing ? launch3<T, C, S, false, 1>(a, coefs, block, s, pdl, npt)
                   : launch3<T, C, S, false, 0>(a, coefs, block, s, pdl, npt);
}

template <typename T, typename C>
static cudaError_t launch1(int n_species, int bc_y, int forcing, const LatticeArgs& a,
                           const void* coefs, dim3 block, cudaStream_t s, bool pdl, int npt) {
    switch (n_species) {
        case 0: return launch2<T, C, 0>(bc_y, forcing, a, coefs, block, s, pdl, npt);
        case 1: return launch2<T, C, 1>(bc_y, forcing, a, coefs, block, s, pdl, npt);
        case 2: return launch2<T, C, 2>(bc_y, forcing, a, coefs, block, s, pdl, npt);
        case 3: return launch2<T, C, 3>(bc_y, forcing, a, coefs, block, s, pdl, npt);
        default: return launch2<T, C, 4>(bc_y, forcing, a, coefs, block, s, pdl, npt);
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
                           bool pdl, int npt) {
    // confined species: the kernels with their paths compiled in
    if (a.dom && n_species > 0)
        return launch_lattice_confined(precision, n_species, bc_y, forcing, a, coefs, block, s,
                                       pdl);
    if (precision == LBIB_FP64)
        return launch1<double, double>(n_species, bc_y, forcing, a, coefs, block, s, pdl, npt);
    if (precision == LBIB_FP32)
        return launch1<float, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl, npt);
    return launch1<__half, float>(n_species, bc_y, forcing, a, coefs, block, s, pdl, npt);
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
