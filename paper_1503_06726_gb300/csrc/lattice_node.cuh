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
// Addresses are a plane base (the same for every thread) plus a 32-bit index
// within the plane (a plane holds fewer than 2^31 elements).
template <typename T, typename C, bool WALLS>
__device__ __forceinline__ void pull5(const T* B, int64_t P, int node, int r0, int rm, int rp,
                                      int x, int xm, int xp, bool lo, bool hi, uint64_t pol,
                                      C g[5]) {
    using St = Store<T, C>;
    g[0] = St::ld(B + node, pol);
    g[1] = St::ld((B + 1 * P) + (r0 + xm), pol);
    g[3] = St::ld((B + 3 * P) + (r0 + xp), pol);
    g[2] = (WALLS && lo) ? St::ld((B + 4 * P) + node, pol) : St::ld((B + 2 * P) + (rm + x), pol);
    g[4] = (WALLS && hi) ? St::ld((B + 2 * P) + node, pol) : St::ld((B + 4 * P) + (rp + x), pol);
}

// The D2Q5 pull of a species confined to its domain (the membrane no-flux
// condition, Sec. 6.1, as half-way bounce-back): a population whose source
// node lies in another domain (label in dom) is the opposite population of
// the node itself, so nothing crosses a domain boundary.
template <typename T, typename C, bool WALLS>
__device__ __forceinline__ void pull5_confined(const T* B, int64_t P, const int32_t* dom,
                                               int node, int r0, int rm, int rp, int x, int xm,
                                               int xp, bool lo, bool hi, uint64_t pol,
                                               C g[5]) {
    using St = Store<T, C>;
    const int32_t d0 = dom[node];
    const bool bl = dom[r0 + xm] != d0, br = dom[r0 + xp] != d0;
    const bool bd = (WALLS && lo) || dom[rm + x] != d0;
    const bool bu = (WALLS && hi) || dom[rp + x] != d0;
    g[0] = St::ld(B + node, pol);
    g[1] = bl ? St::ld((B + 3 * P) + node, pol) : St::ld((B + 1 * P) + (r0 + xm), pol);
    g[3] = br ? St::ld((B + 1 * P) + node, pol) : St::ld((B + 3 * P) + (r0 + xp), pol);
    g[2] = bd ? St::ld((B + 4 * P) + node, pol) : St::ld((B + 2 * P) + (rm + x), pol);
    g[4] = bu ? St::ld((B + 2 * P) + node, pol) : St::ld((B + 4 * P) + (rp + x), pol);
}

// The D2Q5 pull of a species confined by the paper's no-flux closure
// (Sec. 6.1): a population whose source node lies in another domain (bit q
// of the node's code) is the equilibrium w_q (phi^ + v_q.j(y1)) of the
// previous step's moments M (planes phi, jx, jy of the species, compute
// type): phi^ = 2 phi(y1) - phi(y2) extrapolated along the link from
// y1 = x + v_q and y2 = x + 2 v_q, the momentum j(y1)/3 interpolated to zero
// at the half-way wall point (times the 3 of the equilibrium); where y2 (or
// y1) is not in the domain the density comes from y1 (or the node itself,
// with no momentum).  Walls bounce back as in pull5.  In stored units:
// unscaled storage keeps g, FP16 storage g / (w sigma_g) (isg = 1/sigma_g).
// The moments were written by the lattice launch two launches back: read
// through L2.
template <typename T, typename C, bool WALLS, bool SCALED>
__device__ __forceinline__ void pull5_closure(const T* B, int64_t P, const C* M, uint32_t code,
                                              int node, int r0, int rm, int rp, int rmm, int rpp,
                                              int x, int xm, int xp, int xmm, int xpp, bool lo,
                                              bool hi, uint64_t pol, C isg, C wq, C g[5],
                                              uint32_t* diag) {
    using St = Store<T, C>;
    g[0] = St::ld(B + node, pol);
#pragma unroll
    for (int q = 1; q <= 4; ++q) {
        if ((code >> (kNcodeMiss + q - 1)) & 1u) {
            const int i1 = q == 1 ? r0 + xp : (q == 3 ? r0 + xm : (q == 2 ? rp + x : rm + x));
            const int i2 = q == 1 ? r0 + xpp : (q == 3 ? r0 + xmm : (q == 2 ? rpp + x : rmm + x));
            if (!LBIB_CHK_INDEX(diag, kSiteClosureIndex, i1, P) ||
                !LBIB_CHK_INDEX(diag, kSiteClosureIndex, i2, P)) {
                g[q] = C(0);
                continue;
            }
            const bool in1 = (code >> (kNcodeIn1 + q - 1)) & 1u;
            const bool in2 = (code >> (kNcodeIn2 + q - 1)) & 1u;
            const C* Mj = M + (q == 1 || q == 3 ? P : 2 * P);
            C ph, jc;
            if (in1) {
                const C p1 = __ldcg(M + i1);
                const C j1 = __ldcg(Mj + i1);
                ph = in2 ? C(2) * p1 - __ldcg(M + i2) : p1;
                jc = (q == 1 || q == 2) ? j1 : -j1;
            } else {
                ph = __ldcg(M + node);
                jc = C(0);
            }
            g[q] = SCALED ? (ph + jc) * isg : wq * (ph + jc);
        } else if (q == 1) {
            g[1] = St::ld((B + 1 * P) + (r0 + xm), pol);
        } else if (q == 3) {
            g[3] = St::ld((B + 3 * P) + (r0 + xp), pol);
        } else if (q == 2) {
            g[2] = (WALLS && lo) ? St::ld((B + 4 * P) + node, pol)
                                 : St::ld((B + 2 * P) + (rm + x), pol);
        } else {
            g[4] = (WALLS && hi) ? St::ld((B + 2 * P) + node, pol)
                                 : St::ld((B + 4 * P) + (rp + x), pol);
        }
    }
}

// The update of one node (x, y).  Callers map the 32 lanes of a warp to 32
// consecutive nodes of one row starting at a multiple of 32 (lane = x mod
// 32): lane 0 clears the warp's group-mask bits.
// The body is a macro so that the standalone kernel expands it directly on its
// kernel parameters (a separate inlined function measured 17% slower there,
// with identical memory traffic); the ensemble's device function expands the
// same text.  It uses the names a (LatticeArgs), k (Coefs<C>), x, y, the
// template parameters T, C, S, WALLS, FORCING, SCALED and two constexpr
// bools: GRIDDEP, with which the population loads (written by the lattice
// launch two launches back, read through L2) are issued before the
// programmatic wait on the IB kernel whose force, label and mask planes the
// rest reads; CONF, without which the paths of confined species (domain
// planes, the no-flux closure and its moments) are compiled out; OPTS,
// without which the mass sources, node sources and pressure nodes are
// (the ensemble has none of them and keeps its registers).
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
    const int r0 = y * (int)a.pitch; \
    const int rm = ym * (int)a.pitch; \
    const int rp = yp * (int)a.pitch; \
    const int node = r0 + x; \
    /* the checking build: every pulled index inside the plane, the plane */ \
    /* bases aligned to their elements */ \
    if (!LBIB_CHK_INDEX(a.diag, kSiteLatticeIndex, \
                        (int64_t)(rm > rp ? (rm > r0 ? rm : r0) : (rp > r0 ? rp : r0)) + \
                            (xm > xp ? (xm > x ? xm : x) : (xp > x ? xp : x)), \
                        a.plane) || \
        !LBIB_CHK_ACCESS(a.diag, kSiteLatticeAlign, a.fsrc, (int)sizeof(T), nullptr, nullptr) || \
        !LBIB_CHK_ACCESS(a.diag, kSiteLatticeAlign, a.fdst, (int)sizeof(T), nullptr, nullptr) || \
        !LBIB_CHK_ACCESS(a.diag, kSiteLatticeAlign, a.u, (int)sizeof(V2), nullptr, nullptr) || \
        !LBIB_CHK_ACCESS(a.diag, kSiteLatticeAlign, a.force, (int)sizeof(V2), nullptr, nullptr) || \
        !LBIB_CHK_INDEX(a.diag, kSiteMask, (int64_t)(node >> 7), mask_words(a.plane))) \
        return; \
 \
    /* ---- every load of the node first (all independent, read-only path), so */ \
    /* that a thread has all its DRAM requests in flight at once */ \
    const T* F = static_cast<const T*>(a.fsrc); \
    C d[9]; \
    const uint64_t pol = a.l2_first ? l2_evict_first() : l2_evict_normal(); \
    pull5<T, C, WALLS>(F, P, node, r0, rm, rp, x, xm, xp, lo_wall, hi_wall, pol, d); \
    if (lo_wall) {  /* half-way bounce-back: v_y = +1 populations reflect off y = -1/2 */ \
        d[5] = St::ld((F + 7 * P) + node, pol); \
        d[6] = St::ld((F + 8 * P) + node, pol); \
    } else { \
        d[5] = St::ld((F + 5 * P) + (rm + xm), pol); \
        d[6] = St::ld((F + 6 * P) + (rm + xp), pol); \
    } \
    if (hi_wall) {  /* v_y = -1 populations reflect off y = ny - 1/2 */ \
        d[7] = St::ld((F + 5 * P) + node, pol); \
        d[8] = St::ld((F + 6 * P) + node, pol); \
    } else { \
        d[7] = St::ld((F + 7 * P) + (rp + xp), pol); \
        d[8] = St::ld((F + 8 * P) + (rp + xm), pol); \
    } \
    C g[S > 0 ? S : 1][5]; \
    /* confined species: the node's closure code (the paper's no-flux */ \
    /* closure) or its domain (half-way bounce-back) */ \
    uint32_t ncode = 0u; \
    if (CONF && a.ncode) ncode = a.ncode[node]; \
    { \
        const T* Gi = static_cast<const T*>(a.gsrc); \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
            if (CONF && a.dom && ((a.noflux >> s) & 1)) { \
                if (a.ncode) { \
                    const int ypp = (y + 2 >= a.ny) ? y + 2 - a.ny : y + 2; \
                    const int ymm = (y < 2) ? y - 2 + a.ny : y - 2; \
                    const int xpp = (x + 2 >= a.nx) ? x + 2 - a.nx : x + 2; \
                    const int xmm = (x < 2) ? x - 2 + a.nx : x - 2; \
                    pull5_closure<T, C, WALLS, SCALED>( \
                        Gi + (int64_t)s * 5 * P, P, \
                        static_cast<const C*>(a.mom_in) + (int64_t)s * 3 * P, ncode, node, r0, \
                        rm, rp, ymm * (int)a.pitch, ypp * (int)a.pitch, x, xm, xp, xmm, xpp, \
                        lo_wall, hi_wall, pol, k.isig_g, k.w5c[1], g[s], a.diag); \
                } else { \
                    pull5_confined<T, C, WALLS>(Gi + (int64_t)s * 5 * P, P, a.dom, node, r0, rm, \
                                                rp, x, xm, xp, lo_wall, hi_wall, pol, g[s]); \
                } \
            } else { \
                pull5<T, C, WALLS>(Gi + (int64_t)s * 5 * P, P, node, r0, rm, rp, x, xm, xp, \
                                   lo_wall, hi_wall, pol, g[s]); \
            } \
        } \
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
    const int grp = node >> 2; \
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
    /* ---- the collision (collide_node), then the stores */ \
    C rho, ux, uy; \
    C ph[S > 0 ? S : 1]; \
    /* the cell's mass source at labelled nodes; internal pressure nodes */ \
    C ms = C(0); \
    if (OPTS && a.msrc && label != kOutside) ms = static_cast<const C*>(a.msrc)[label >> 4]; \
    if (OPTS && a.nsrc) ms += static_cast<const C*>(a.nsrc)[node]; \
    const bool pn = OPTS && a.pnode && a.pnode[node] != 0; \
    /* the closure reads this node's moments next step: its species fluxes */ \
    /* before the collision (the densities come out of collide_node) */ \
    const bool mom_w = CONF && ((ncode >> kNcodeMom) & 1u); \
    C mjx[S > 0 ? S : 1], mjy[S > 0 ? S : 1]; \
    if (mom_w) { \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
            const C gs = SCALED ? k.gscale[1] : C(1); \
            mjx[s] = gs * (g[s][1] - g[s][3]); \
            mjy[s] = gs * (g[s][2] - g[s][4]); \
        } \
    } \
    collide_node<C, S, FORCING, SCALED>(k, d, g, fv.x, fv.y, sbits, 0u, rho, ux, uy, ph, \
                                        OPTS && (a.msrc != nullptr || a.nsrc != nullptr), ms, \
                                        pn); \
    if (mom_w) { \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
            if ((a.noflux >> s) & 1) { \
                C* Mo = static_cast<C*>(a.mom_out) + (int64_t)s * 3 * P; \
                Mo[node] = ph[s]; \
                (Mo + P)[node] = mjx[s]; \
                (Mo + 2 * P)[node] = mjy[s]; \
            } \
        } \
    } \
    T* G = static_cast<T*>(a.fdst); \
_Pragma("unroll") \
    for (int q = 0; q < 9; ++q) St::st((G + q * P) + node, d[q]); \
    if (S > 0) { \
        T* Go = static_cast<T*>(a.gdst); \
_Pragma("unroll") \
        for (int s = 0; s < S; ++s) { \
_Pragma("unroll") \
            for (int q = 0; q < 5; ++q) St::st((Go + (int64_t)(s * 5 + q) * P) + node, g[s][q]); \
            if (a.out) (static_cast<C*>(a.phi) + (int64_t)s * P)[node] = ph[s]; \
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

// Explicit round-to-nearest operations on the value of one node (float,
// double) or of two nodes at once (float2: the packed FP32 instructions of
// sm_100 and later, which per component are the float operation).  The
// collision is written with them, so a node gets bit-identical results
// whichever form evaluates it, and the compiler neither re-associates nor
// contracts it.
template <typename V>
struct Lane;
template <>
struct Lane<float> {
    using S = float;
    static __device__ __forceinline__ float c(float s) { return s; }
    static __device__ __forceinline__ float sel(bool a, bool, float v) { return a ? v : 0.f; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) {
        return __fmaf_rn(a, b, c);
    }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
};
template <>
struct Lane<float2> {
    using S = float;
    static __device__ __forceinline__ float2 c(float s) { return make_float2(s, s); }
    static __device__ __forceinline__ float2 sel(bool a, bool b, float v) {
        return make_float2(a ? v : 0.f, b ? v : 0.f);
    }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) {
        return __fadd2_rn(a, make_float2(-b.x, -b.y));
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) {
        return __ffma2_rn(a, b, c);
    }
    static __device__ __forceinline__ float2 rcp(float2 a) {
        return make_float2(__frcp_rn(a.x), __frcp_rn(a.y));
    }
};
template <>
struct Lane<double> {
    using S = double;
    static __device__ __forceinline__ double c(double s) { return s; }
    static __device__ __forceinline__ double sel(bool a, bool, double v) { return a ? v : 0.0; }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) {
        return __fma_rn(a, b, c);
    }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
};

// The collision of one node (or two, V = float2) in registers, Sec. 6.1 in
// deviation form:
//   rho = rho0 + sum d,  u = (sum d v + F/2) / rho  (Guo; the paper's term: no F/2)
//   with A = omega drho, W = omega rho, for a direction q and its opposite q':
//   d*_q  = (1 - omega) d_q  + w (E + 3 W v.u + Co)
//   d*_q' = (1 - omega) d_q' + w (E - 3 W v.u - Co)
//   E = A + W (9/2 (v.u)^2 - 3/2 u.u) + Ce
//   Guo: Ce = pref (9 (v.u)(v.F) - 3 u.F), Co = 3 pref v.F;  paper: Ce = 0, Co = 3 v.F
// and every species (D2Q5) with phi = sum g, R = reaction + source:
//   g*_q = (1 - omega_D) g_q + w (omega_D phi + R) + w 3 omega_D phi v.u
// Scaled storage (FP16) keeps s_q = d_q / (w_q sigma): the moments weight the
// stored values and 1/sigma replaces w.  d and g enter as the pulled stored
// values and leave as the post-collision stored values; bitsA / bitsB are the
// source bits of the node(s).
template <typename V, int S, int FORCING, bool SCALED>
__device__ __forceinline__ void collide_node(const Coefs<typename Lane<V>::S>& k, V (&d)[9],
                                             V (&g)[S > 0 ? S : 1][5], V fvx, V fvy,
                                             uint32_t bitsA, uint32_t bitsB, V& rho, V& ux,
                                             V& uy, V (&ph)[S > 0 ? S : 1],
                                             bool mass_on = false, V ms = V(),
                                             bool pnode = false) {
    using L = Lane<V>;
    using C = typename L::S;
    const V Fx = L::add(L::c(k.bfx), fvx), Fy = L::add(L::c(k.bfy), fvy);
    V drho, jx, jy;
    if (SCALED) {
        const V sB = L::c(k.fscale[1]), sC = L::c(k.fscale[5]);
        const V a14 = L::add(L::add(d[1], d[2]), L::add(d[3], d[4]));
        const V a58 = L::add(L::add(d[5], d[6]), L::add(d[7], d[8]));
        drho = L::fma(L::c(k.fscale[0]), d[0], L::fma(sB, a14, L::mul(sC, a58)));
        jx = L::fma(sB, L::sub(d[1], d[3]),
                    L::mul(sC, L::add(L::sub(d[5], d[6]), L::sub(d[8], d[7]))));
        jy = L::fma(sB, L::sub(d[2], d[4]),
                    L::mul(sC, L::sub(L::add(d[5], d[6]), L::add(d[7], d[8]))));
    } else {
        drho = L::add(L::add(L::add(L::add(d[0], d[1]), L::add(d[2], d[3])),
                             L::add(L::add(d[4], d[5]), L::add(d[6], d[7]))),
                      d[8]);
        jx = L::add(L::add(L::sub(d[1], d[3]), L::sub(d[5], d[6])), L::sub(d[8], d[7]));
        jy = L::sub(L::add(L::sub(d[2], d[4]), L::add(d[5], d[6])), L::add(d[7], d[8]));
    }
    if (pnode) {
        // internal pressure node (Sec. 6.1): every population scaled by
        // gamma = rho_p / rho, so the node holds rho_p and keeps u; on the
        // deviations d = f - w rho0 (scaled: / (w sigma)) that is
        // d <- gamma d + (gamma - 1) w rho0 (scaled: (gamma - 1) rho0 / sigma)
        const V gam = L::mul(L::c(k.prho), L::rcp(L::add(L::c(k.rho0), drho)));
        const V gm1 = L::sub(gam, L::c(C(1)));
#pragma unroll
        for (int q = 0; q < 9; ++q)
            d[q] = L::fma(gam, d[q], L::mul(gm1, L::c(SCALED ? k.rho0 * k.isig : k.w9c[q == 0 ? 0 : (q < 5 ? 1 : 2)] * k.rho0)));
        drho = L::c(k.prho - k.rho0);
        jx = L::mul(gam, jx);
        jy = L::mul(gam, jy);
    }
    rho = L::add(L::c(k.rho0), drho);
    const V irho = L::rcp(rho);
    if (FORCING == LBIB_GUO) {
        ux = L::mul(L::fma(L::c(C(0.5)), Fx, jx), irho);
        uy = L::mul(L::fma(L::c(C(0.5)), Fy, jy), irho);
    } else {
        ux = L::mul(jx, irho);
        uy = L::mul(jy, irho);
    }
    const V nusq = L::mul(L::c(C(-1.5)), L::fma(ux, ux, L::mul(uy, uy)));  // -3/2 u.u
    const V A = L::mul(L::c(k.omega), drho);
    const V W = L::mul(L::c(k.omega), rho);
    const V W3 = L::mul(L::c(C(3)), W);
    const V W45 = L::mul(L::c(C(4.5)), W);
    V E0 = L::fma(W, nusq, A);  // the even part common to every direction
    if (FORCING == LBIB_GUO)
        E0 = L::fma(L::c(C(-3) * k.pref), L::fma(ux, Fx, L::mul(uy, Fy)), E0);
    // mass source (Sec. 3.2.3): w_q S added to every direction, no momentum
    if (mass_on) E0 = L::add(E0, ms);
    const V omc = L::c(k.omc);
    d[0] = L::fma(L::c(SCALED ? k.isig : k.w9c[0]), E0, L::mul(omc, d[0]));
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        if (q == 1 || q == 2 || q == 5 || q == 6) {
            const int o = q + 2;  // opposite of 1, 2, 5, 6
            const V ew = L::c(SCALED ? k.isig : k.w9c[q < 5 ? 1 : 2]);
            // v.u and v.F of v = (1,0), (0,1), (1,1), (-1,1)
            const V cu = q == 1 ? ux : (q == 2 ? uy : (q == 5 ? L::add(ux, uy) : L::sub(uy, ux)));
            const V cF = q == 1 ? Fx : (q == 2 ? Fy : (q == 5 ? L::add(Fx, Fy) : L::sub(Fy, Fx)));
            V ev = L::fma(W45, L::mul(cu, cu), E0);
            V od = L::mul(W3, cu);
            if (FORCING == LBIB_GUO) {
                ev = L::fma(L::c(C(9) * k.pref), L::mul(cu, cF), ev);
                od = L::fma(L::c(C(3) * k.pref), cF, od);
            } else {
                od = L::fma(L::c(C(3)), cF, od);
            }
            const V dq = L::fma(ew, L::add(ev, od), L::mul(omc, d[q]));
            const V dqo = L::fma(ew, L::sub(ev, od), L::mul(omc, d[o]));
            d[q] = dq;
            d[o] = dqo;
        }
    }
    if (S > 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (SCALED)
                ph[s] = L::fma(L::c(k.gscale[0]), g[s][0],
                               L::mul(L::c(k.gscale[1]),
                                      L::add(L::add(g[s][1], g[s][2]), L::add(g[s][3], g[s][4]))));
            else
                ph[s] = L::add(L::add(L::add(g[s][0], g[s][1]), L::add(g[s][2], g[s][3])),
                               g[s][4]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            V R = L::sel((bitsA >> s) & 1u, (bitsB >> s) & 1u, k.srate[s]);
            if (S >= 2 && s < 2 && k.react_model == LBIB_REACT_SCHNAKENBERG) {
                // receptor R = species 0, ligand L = species 1 (Sec. 4.2):
                // gamma (a - R + R^2 L) and gamma (b - R^2 L)
                const V r2l = L::mul(L::mul(ph[0], ph[0]), ph[1]);
                const V rate = s == 0 ? L::add(L::sub(L::c(k.sa), ph[0]), r2l)
                                      : L::sub(L::c(k.sb), r2l);
                R = L::fma(L::c(k.sgamma), rate, R);
            } else {
#pragma unroll
                for (int b = 0; b < S; ++b) R = L::fma(L::c(k.K[s][b]), ph[b], R);
            }
            const V ev = L::fma(L::c(k.omegaD[s]), ph[s], R);
            const C eA = SCALED ? k.isig_g : k.w5c[0];
            const C eB = SCALED ? k.isig_g : k.w5c[1];
            const V evB = L::mul(L::c(eB), ev);
            const V o3 = L::mul(L::c(C(3) * eB * k.omegaD[s]), ph[s]);
            const V ox = L::mul(o3, ux), oy = L::mul(o3, uy);
            const V omcD = L::c(k.omcD[s]);
            g[s][0] = L::fma(L::c(eA), ev, L::mul(omcD, g[s][0]));
            g[s][1] = L::fma(omcD, g[s][1], L::add(evB, ox));
            g[s][3] = L::fma(omcD, g[s][3], L::sub(evB, ox));
            g[s][2] = L::fma(omcD, g[s][2], L::add(evB, oy));
            g[s][4] = L::fma(omcD, g[s][4], L::sub(evB, oy));
        }
    }
}

// WAIT: the caller is a kernel of its own, launched programmatically after an
// IB launch (the ensemble's split schedule), with the population loads issued
// before the wait as in the standalone kernel; without it the caller orders
// the phases itself (the persistent kernel's grid barriers).
template <typename T, typename C, int S, bool WALLS, int FORCING, bool SCALED, bool WAIT = false>
__device__ __forceinline__ void lattice_node(const LatticeArgs& a, const Coefs<C>& k, int x,
                                             int y) {
    constexpr bool GRIDDEP = WAIT;
    // the ensemble's tissues confine no species and have no mass sources,
    // node sources or pressure nodes
    constexpr bool CONF = false;
    constexpr bool OPTS = false;
    LBIB_LATTICE_NODE_BODY
}

}  // namespace lbib
