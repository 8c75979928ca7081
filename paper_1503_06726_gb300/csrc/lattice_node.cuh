// lattice_node.cuh -- the fused lattice update of one node (device code
// shared by the per-tissue kernel and the ensemble's persistent kernel).
#pragma once

#include <type_traits>

#include "lbib_internal.cuh"

namespace lbib {


template <typename T, typename C>
struct Store;
template <>
struct Store<double, double> {
    static __device__ __forceinline__ double ld(const double* p, uint64_t pol) {
        return ld_stream(p, pol);
    }
    static __device__ __forceinline__ void st(double* p, double v) { *p = v; }
};
template <>
struct Store<float, float> {
    static __device__ __forceinline__ float ld(const float* p, uint64_t pol) {
        return ld_stream(p, pol);
    }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Store<__half, float> {
    static __device__ __forceinline__ float ld(const __half* p, uint64_t pol) {
        return __half2float(
            __ushort_as_half(ld_stream(reinterpret_cast<const unsigned short*>(p), pol)));
    }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};

template <typename C>
struct Vec2;
template <>
struct Vec2<double> { using T = double2; };
template <>
struct Vec2<float> { using T = float2; };

// Pull the 5 populations of one D2Q5 set (or the first 5 of D2Q9) at a node.
template <typename T, typename C, bool WALLS>
__device__ __forceinline__ void pull5(const T* B, int64_t P, int64_t node, int64_t r0, int64_t rm,
                                      int64_t rp, int x, int xm, int xp, bool lo, bool hi,
                                      uint64_t pol, C g[5]) {
    using St = Store<T, C>;
    g[0] = St::ld(B + node, pol);
    g[1] = St::ld(B + 1 * P + r0 + xm, pol);
    g[3] = St::ld(B + 3 * P + r0 + xp, pol);
    g[2] = (WALLS && lo) ? St::ld(B + 4 * P + node, pol) : St::ld(B + 2 * P + rm + x, pol);
    g[4] = (WALLS && hi) ? St::ld(B + 2 * P + node, pol) : St::ld(B + 4 * P + rp + x, pol);
}

// The update of one node (x, y).  Callers map the 32 lanes of a warp to 32
// consecutive nodes of one row starting at a multiple of 32 (lane = x mod
// 32): lane 0 clears the warp's group-mask bits.
// The body is a macro so that the standalone kernel expands it directly on its
// kernel parameters (a separate inlined function measured 17% slower there,
// with identical memory traffic); the ensemble's device function expands the
// same text.  It uses the names a (LatticeArgs), k (Coefs<C>), x, y, the
// template parameters T, C, S, WALLS, FORCING, SCALED and a constexpr bool
// GRIDDEP: with it the population loads (written by the lattice launch two
// launches back, read through L2) are issued before the programmatic wait on
// the IB kernel whose force, label and mask planes the rest reads.
#define LBIB_LATTICE_NODE_BODY \
 \
    using St = Store<T, C>; \
    using V2 = typename Vec2<C>::T; \
 \
    const int64_t P = a.plane; \
    const int xm = (x == 0) ? a.nx - 1 : x - 1; \
    const int xp = (x == a.nx - 1) ? 0 : x + 1; \
    const bool lo_wall = WALLS && (y == 0); \
    const bool hi_wall = WALLS && (y == a.ny - 1); \
    const int ym = (y == 0) ? a.ny - 1 : y - 1; \
    const int yp = (y == a.ny - 1) ? 0 : y + 1; \
    const int64_t r0 = (int64_t)y * a.pitch; \
    const int64_t rm = (int64_t)ym * a.pitch; \
    const int64_t rp = (int64_t)yp * a.pitch; \
    const int64_t node = r0 + x; \
 \
    /* ---- every load of the node first (all independent, read-only path), so */ \
    /* that a thread has all its DRAM requests in flight at once */ \
    const T* F = static_cast<const T*>(a.fsrc); \
    C d[9]; \
    const uint64_t pol = a.l2_first ? l2_evict_first() : l2_evict_normal(); \
    pull5<T, C, WALLS>(F, P, node, r0, rm, rp, x, xm, xp, lo_wall, hi_wall, pol, d); \
    if (lo_wall) {  /* half-way bounce-back: v_y = +1 populations reflect off y = -1/2 */ \
        d[5] = St::ld(F + 7 * P + node, pol); \
        d[6] = St::ld(F + 8 * P + node, pol); \
    } else { \
        d[5] = St::ld(F + 5 * P + rm + xm, pol); \
        d[6] = St::ld(F + 6 * P + rm + xp, pol); \
    } \
    if (hi_wall) {  /* v_y = -1 populations reflect off y = ny - 1/2 */ \
        d[7] = St::ld(F + 5 * P + node, pol); \
        d[8] = St::ld(F + 6 * P + node, pol); \
    } else { \
        d[7] = St::ld(F + 7 * P + rp + xp, pol); \
        d[8] = St::ld(F + 8 * P + rp + xm, pol); \
    } \
    C g[S > 0 ? S : 1][5]; \
    { \
        const T* Gi = static_cast<const T*>(a.gsrc); \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) \
            pull5<T, C, WALLS>(Gi + (int64_t)s * 5 * P, P, node, r0, rm, rp, x, xm, xp, lo_wall, \
                               hi_wall, pol, g[s]); \
    } \
    /* the IB kernel launched just before wrote the force, label and mask */ \
    /* planes: wait for it, then let the next IB launch start */ \
    if (GRIDDEP) { \
        griddep_wait(); \
        griddep_launch_dependents(); \
    } \
    /* spread force, labels and source bits: only the 4-node groups the IB */ \
    /* kernel marked (labels are written only before an output step) */ \
    V2 fv; \
    fv.x = C(0); \
    fv.y = C(0); \
    uint32_t label = kOutside, sbits = 0u; \
    bool fhit = false, lhit = false, shit = false; \
    /* for lane 0: which masks hold bits of this warp's 8 groups */ \
    uint32_t clear = 0u; \
    const int64_t grp = node >> 2; \
    if (a.ib) { \
        if (a.fmask) { \
            const int sh = (int)(grp & 31); \
            const uint32_t fw = a.fmask[grp >> 5] >> sh; \
            const uint32_t lw = a.lmask[grp >> 5] >> sh; \
            const uint32_t sw = a.smask[grp >> 5] >> sh; \
            fhit = fw & 1u; \
            lhit = lw & 1u; \
            shit = sw & 1u; \
            clear = ((fw & 0xFFu) ? 1u : 0u) | ((lw & 0xFFu) ? 2u : 0u) | \
                    ((sw & 0xFFu) ? 4u : 0u); \
        } else { \
            fhit = shit = true; \
            lhit = a.id != nullptr; \
        } \
        if (fhit) fv = static_cast<const V2*>(a.force)[node]; \
        if (lhit) label = a.id[node]; \
        if (shit) sbits = a.src[node]; \
    } \
 \
    /* ---- moments (Sec. 6.1) with the half-force velocity shift (Guo).  With */ \
    /* scaled storage s_q = d_q / (w_q sigma) the moments weight the stored */ \
    /* values (w_1..w_4 and w_5..w_8 are equal) and d_q is never formed. */ \
    const C Fx = k.bfx + fv.x, Fy = k.bfy + fv.y; \
    C drho, jx, jy; \
    if (SCALED) { \
        const C sA = k.fscale[0], sB = k.fscale[1], sC = k.fscale[5]; \
        drho = sA * d[0] + sB * ((d[1] + d[2]) + (d[3] + d[4])) + \
               sC * ((d[5] + d[6]) + (d[7] + d[8])); \
        jx = sB * (d[1] - d[3]) + sC * ((d[5] - d[6]) + (d[8] - d[7])); \
        jy = sB * (d[2] - d[4]) + sC * ((d[5] + d[6]) - (d[7] + d[8])); \
    } else { \
        drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8]; \
        jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]); \
        jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]); \
    } \
    const C rho = k.rho0 + drho; \
    const C irho = C(1) / rho; \
    C ux, uy; \
    if (FORCING == LBIB_GUO) { \
        ux = (jx + C(0.5) * Fx) * irho; \
        uy = (jy + C(0.5) * Fy) * irho; \
    } else { \
        ux = jx * irho; \
        uy = jy * irho; \
    } \
    const C usq15 = C(1.5) * (ux * ux + uy * uy); \
    const C uF = ux * Fx + uy * Fy; \
 \
    /* ---- collide and store the fluid, opposite directions together: with */ \
    /* A = drho + rho (9/2 (v.u)^2 - 3/2 u.u), B = 3 rho v.u and the forcing */ \
    /* split into its even part Ce and odd part Co, */ \
    /*   d*_q = (1 - omega) d_q + w (omega A + Ce) + w (omega B + Co) */ \
    /* and the opposite direction flips the sign of the odd terms.  Scaled */ \
    /* storage replaces the factor w by 1/sigma. */ \
    T* G = static_cast<T*>(a.fdst); \
    { \
        const C e0 = SCALED ? k.isig : C(w9(0)); \
        C ev = k.omega * (drho - rho * usq15); \
        if (FORCING == LBIB_GUO) ev -= k.pref * (C(3) * uF); \
        St::st(G + node, k.omc * d[0] + e0 * ev); \
    } \
_Pragma("unroll") \
    for (int q = 1; q < 9; ++q) { \
        if (q == 1 || q == 2 || q == 5 || q == 6) { \
            const int o = q + 2; /* opposite of 1, 2, 5, 6 */ \
            const C ew = SCALED ? k.isig : C(w9(q)); \
            const C cu = C(cx(q)) * ux + C(cy(q)) * uy; \
            const C cF = C(cx(q)) * Fx + C(cy(q)) * Fy; \
            C ev = k.omega * (drho + rho * (C(4.5) * cu * cu - usq15)); \
            C od = k.omega * (rho * (C(3) * cu)); \
            if (FORCING == LBIB_GUO) { \
                ev += k.pref * (C(9) * cu * cF - C(3) * uF); \
                od += k.pref * (C(3) * cF); \
            } else { \
                od += C(3) * cF; \
            } \
            ev *= ew; \
            od *= ew; \
            St::st(G + q * P + node, k.omc * d[q] + (ev + od)); \
            St::st(G + o * P + node, k.omc * d[o] + (ev - od)); \
        } \
    } \
 \
    /* ---- species (D2Q5): react and collide with the fluid u, opposite */ \
    /* directions together: g*_q = (1 - omega_D) g_q + w (omega_D phi + R) */ \
    /* + w omega_D phi 3 v.u (scaled storage: 1/sigma_g for w) */ \
    if (S > 0) { \
        const uint32_t bits = sbits & 0xFu; \
        T* Go = static_cast<T*>(a.gdst); \
        C ph[S > 0 ? S : 1]; \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
            if (SCALED) \
                ph[s] = k.gscale[0] * g[s][0] + \
                        k.gscale[1] * ((g[s][1] + g[s][2]) + (g[s][3] + g[s][4])); \
            else \
                ph[s] = ((g[s][0] + g[s][1]) + (g[s][2] + g[s][3])) + g[s][4]; \
        } \
        const C cux = ux, cuy = uy; \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
            C R = ((bits >> s) & 1u) ? k.srate[s] : C(0); \
_Pragma("unroll") \
            for (int b = 0; b < S; ++b) R += k.K[s][b] * ph[b]; \
            T* B = Go + (int64_t)s * 5 * P; \
            const C ev = k.omegaD[s] * ph[s] + R; \
            const C od = k.omegaD[s] * ph[s] * C(3); \
            const C eA = SCALED ? k.isig_g : C(w5(0)); \
            const C eB = SCALED ? k.isig_g : C(w5(1)); \
            const C evB = eB * ev; \
            const C ox = eB * od * cux, oy = eB * od * cuy; \
            St::st(B + node, k.omcD[s] * g[s][0] + eA * ev); \
            St::st(B + 1 * P + node, k.omcD[s] * g[s][1] + (evB + ox)); \
            St::st(B + 3 * P + node, k.omcD[s] * g[s][3] + (evB - ox)); \
            St::st(B + 2 * P + node, k.omcD[s] * g[s][2] + (evB + oy)); \
            St::st(B + 4 * P + node, k.omcD[s] * g[s][4] + (evB - oy)); \
            if (a.out) static_cast<C*>(a.phi)[(int64_t)s * P + node] = ph[s]; \
        } \
    } \
 \
    /* ---- velocity where the interpolation will read it (the groups that */ \
    /* received force: the kernel support of the same vertex positions) or */ \
    /* everywhere on an output step; resets (after the compute: stores placed */ \
    /* before it measured 3x slower); outputs; the group masks */ \
    if (a.out || fhit) { \
        V2 uv; \
        uv.x = ux; \
        uv.y = uy; \
        st_keep(static_cast<V2*>(a.u) + node, uv); \
    } \
    if (a.ib) { \
        if (fhit) { \
            V2 z; \
            z.x = C(0); \
            z.y = C(0); \
            st_keep(static_cast<V2*>(a.force) + node, z); \
        } \
        if (lhit) a.id[node] = kOutside; \
        if (shit) a.src[node] = 0; \
        if (a.out) { \
            a.id_out[node] = label; \
            static_cast<V2*>(a.force_out)[node] = fv; \
        } \
        /* lane 0 clears the warp's 8 group bits (32 nodes, one row, 32-aligned) */ \
        if (clear && (threadIdx.x & 31) == 0) { \
            const int sh = (int)(grp & 31); \
            if (clear & 1u) atomicAnd(a.fmask + (grp >> 5), ~(0xFFu << sh)); \
            if (clear & 2u) atomicAnd(a.lmask + (grp >> 5), ~(0xFFu << sh)); \
            if (clear & 4u) atomicAnd(a.smask + (grp >> 5), ~(0xFFu << sh)); \
        } \
    } \
    if (a.out) static_cast<C*>(a.rho)[node] = rho; \
    if (!(rho > C(0)) || !isfinite(ux) || !isfinite(uy)) atomicOr(a.diag + kDiagNonFinite, 1u);

// The collision of one node in registers: the arithmetic of the fused update
// above, operation for operation, without its loads and stores.  d and g hold
// the pulled populations in their stored form and are overwritten with the
// post-collision stored values; rho, u and the species fields are returned.
template <typename C, int S, int FORCING, bool SCALED>
__device__ __forceinline__ void collide_node(const Coefs<C>& k, C (&d)[9],
                                             C (&g)[S > 0 ? S : 1][5], C fvx, C fvy,
                                             uint32_t sbits, C& rho, C& ux, C& uy,
                                             C (&ph)[S > 0 ? S : 1]) {
    const C Fx = k.bfx + fvx, Fy = k.bfy + fvy;
    C drho, jx, jy;
    if (SCALED) {
        const C sA = k.fscale[0], sB = k.fscale[1], sC = k.fscale[5];
        drho = sA * d[0] + sB * ((d[1] + d[2]) + (d[3] + d[4])) +
               sC * ((d[5] + d[6]) + (d[7] + d[8]));
        jx = sB * (d[1] - d[3]) + sC * ((d[5] - d[6]) + (d[8] - d[7]));
        jy = sB * (d[2] - d[4]) + sC * ((d[5] + d[6]) - (d[7] + d[8]));
    } else {
        drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    }
    rho = k.rho0 + drho;
    const C irho = C(1) / rho;
    if (FORCING == LBIB_GUO) {
        ux = (jx + C(0.5) * Fx) * irho;
        uy = (jy + C(0.5) * Fy) * irho;
    } else {
        ux = jx * irho;
        uy = jy * irho;
    }
    const C usq15 = C(1.5) * (ux * ux + uy * uy);
    const C uF = ux * Fx + uy * Fy;
    {
        const C e0 = SCALED ? k.isig : C(w9(0));
        C ev = k.omega * (drho - rho * usq15);
        if (FORCING == LBIB_GUO) ev -= k.pref * (C(3) * uF);
        d[0] = k.omc * d[0] + e0 * ev;
    }
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        if (q == 1 || q == 2 || q == 5 || q == 6) {
            const int o = q + 2;
            const C ew = SCALED ? k.isig : C(w9(q));
            const C cu = C(cx(q)) * ux + C(cy(q)) * uy;
            const C cF = C(cx(q)) * Fx + C(cy(q)) * Fy;
            C ev = k.omega * (drho + rho * (C(4.5) * cu * cu - usq15));
            C od = k.omega * (rho * (C(3) * cu));
            if (FORCING == LBIB_GUO) {
                ev += k.pref * (C(9) * cu * cF - C(3) * uF);
                od += k.pref * (C(3) * cF);
            } else {
                od += C(3) * cF;
            }
            ev *= ew;
            od *= ew;
            const C dq = k.omc * d[q] + (ev + od);
            const C doo = k.omc * d[o] + (ev - od);
            d[q] = dq;
            d[o] = doo;
        }
    }
    if (S > 0) {
        const uint32_t bits = sbits & 0xFu;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (SCALED)
                ph[s] = k.gscale[0] * g[s][0] +
                        k.gscale[1] * ((g[s][1] + g[s][2]) + (g[s][3] + g[s][4]));
            else
                ph[s] = ((g[s][0] + g[s][1]) + (g[s][2] + g[s][3])) + g[s][4];
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            C R = ((bits >> s) & 1u) ? k.srate[s] : C(0);
#pragma unroll
            for (int b = 0; b < S; ++b) R += k.K[s][b] * ph[b];
            const C ev = k.omegaD[s] * ph[s] + R;
            const C od = k.omegaD[s] * ph[s] * C(3);
            const C eA = SCALED ? k.isig_g : C(w5(0));
            const C eB = SCALED ? k.isig_g : C(w5(1));
            const C evB = eB * ev;
            const C ox = eB * od * ux, oy = eB * od * uy;
            g[s][0] = k.omcD[s] * g[s][0] + eA * ev;
            g[s][1] = k.omcD[s] * g[s][1] + (evB + ox);
            g[s][3] = k.omcD[s] * g[s][3] + (evB - ox);
            g[s][2] = k.omcD[s] * g[s][2] + (evB + oy);
            g[s][4] = k.omcD[s] * g[s][4] + (evB - oy);
        }
    }
}

template <typename T, typename C, int S, bool WALLS, int FORCING, bool SCALED>
__device__ __forceinline__ void lattice_node(const LatticeArgs a, const Coefs<C> k, int x,
                                             int y) {
    constexpr bool GRIDDEP = false;
    LBIB_LATTICE_NODE_BODY
}

}  // namespace lbib
