// ib_cell.cuh -- device code of the immersed-boundary work of one cell
// (shared by the per-tissue kernels and the ensemble's persistent kernel).
#pragma once

#include <climits>
#include <type_traits>

#include "lbib_internal.cuh"

namespace lbib {


constexpr int kIBThreads = 256;  // CTA of the FP64 path and the persistent ensemble
static_assert(kIBThreads >= kMaxRows, "row counters are cleared one per thread");

__device__ __forceinline__ int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Weights of the 4 support nodes along one axis, base = floor(X) - 1.
// With f = X - floor(X) the four offsets are r = -1-f, -f, 1-f, 2-f, and
// cos(pi |r| / 2) is -sin, cos, sin, -cos of pi f / 2 respectively, so one
// sincospi gives all four values of Eq. 1Dkernel.
template <typename C>
__device__ __forceinline__ void axis_weights(double X, int* base, C w[4]) {
    const double fl = floor(X);
    *base = (int)fl - 1;
    C sn, cs;
    if (sizeof(C) == 8) {
        double s2, c2;
        sincospi(0.5 * (X - fl), &s2, &c2);
        sn = (C)s2;
        cs = (C)c2;
    } else {
        float s2, c2;
        sincospif(0.5f * (float)(X - fl), &s2, &c2);
        sn = (C)s2;
        cs = (C)c2;
    }
    w[0] = C(0.25) * (C(1) - sn);
    w[1] = C(0.25) * (C(1) + cs);
    w[2] = C(0.25) * (C(1) + sn);
    w[3] = C(0.25) * (C(1) - cs);
}

// Cell junction force on a vertex at X with partner vertex j (Eq.
// celljunctionforce): k (d/|d|)(|d| - l0) for d = X_j - X (periodic minimum
// image), zero without a partner or beyond l_max.  The partner's position is
// read from the vertex array, so the calling launch must not be moving the
// vertices.
__device__ __forceinline__ double2 junction_d(const IBArgs& a, double2 X, int j) {
    const double2 Xj = a.xy[j];
    const double dx = min_image(__dsub_rn(Xj.x, X.x), a.nx);
    double dy = __dsub_rn(Xj.y, X.y);
    if (!a.bc_y) dy = min_image(dy, a.ny);
    return make_double2(dx, dy);
}
__device__ __forceinline__ float2 junction_force32(const IBArgs& a, double2 X, int j) {
    if (j < 0) return make_float2(0.f, 0.f);
    const double2 d = junction_d(a, X, j);
    const float dx = (float)d.x, dy = (float)d.y;
    const float L = sqrtf(dx * dx + dy * dy);
    if (!(L < (float)a.jlmax) || !(L > 0.f)) return make_float2(0.f, 0.f);
    const float s = (float)a.jk * (L - (float)a.jl0) / L;
    return make_float2(s * dx, s * dy);
}
__device__ __forceinline__ double2 junction_force64(const IBArgs& a, double2 X, int j) {
    if (j < 0) return make_double2(0.0, 0.0);
    const double2 d = junction_d(a, X, j);
    const double L = sqrt(d.x * d.x + d.y * d.y);
    if (!(L < a.jlmax) || !(L > 0.0)) return make_double2(0.0, 0.0);
    return make_double2(a.jk * d.x / L * (L - a.jl0), a.jk * d.y / L * (L - a.jl0));
}

// Shoelace area of a polygon held in shared memory, taken about its first
// vertex (Sec. 3.3), summed by one warp in FP64; every lane returns it.
__device__ __forceinline__ double cell_area_warp(const double2* sx, int n, int lane) {
    const double2 X0 = sx[0];
    double acc = 0.0;
    for (int t = lane; t < n; t += 32) {
        const double2 A = sx[t], B = sx[t + 1 == n ? 0 : t + 1];
        const double xl = A.x - X0.x, yl = A.y - X0.y, xm = B.x - X0.x, ym = B.y - X0.y;
        acc += xl * ym - xm * yl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return 0.5 * acc;
}

// the mass source of cell c for the step (Sec. 3.2.3): the constant rate plus
// the proportional area controller when target areas are set
__device__ __forceinline__ double mass_source(const IBArgs& a, int c, double area) {
    const double r = a.mrate ? a.mrate[c] : 0.0;
    return a.marea ? r + a.malpha * (a.marea[c] - area) : r;
}

// raise a diagnostic flag (labelling-only callers may pass no flag words)
__device__ __forceinline__ void raise_flag(uint32_t* diag, int k) {
    if (diag) atomicOr(diag + k, 1u);
}

// spread one weighted force into a node: FP32 uses the float2 vector atomic
__device__ __forceinline__ void spread_add(const IBArgs& a, float2* p, float fx, float fy) {
    const float2* f = static_cast<const float2*>(a.force);
    if (LBIB_CHK_ACCESS(a.diag, kSiteIbForce, p, 8, f, f + a.plane)) red_keep(p, fx, fy);
}
__device__ __forceinline__ void spread_add(const IBArgs& a, double2* p, double fx, double fy) {
    const double2* f = static_cast<const double2*>(a.force);
    if (LBIB_CHK_ACCESS(a.diag, kSiteIbForce, p, 16, f, f + a.plane)) {
        atomicAdd(&p->x, fx);
        atomicAdd(&p->y, fy);
    }
}

// The FP32 path's vector accesses to the force and velocity planes, with the
// checking build's tests (address inside the plane, aligned to the access).
__device__ __forceinline__ bool force_ok(const IBArgs& a, const float2* p, int bytes) {
    const float2* f = static_cast<const float2*>(a.force);
    return LBIB_CHK_ACCESS(a.diag, kSiteIbForce, p, bytes, f, f + a.plane);
}
__device__ __forceinline__ void force_red1(const IBArgs& a, float2* p, float x, float y) {
    if (force_ok(a, p, 8)) red_keep(p, x, y);
}
__device__ __forceinline__ void force_red2(const IBArgs& a, float2* p, float x0, float y0,
                                           float x1, float y1) {
    if (force_ok(a, p, 16)) red_keep2(p, x0, y0, x1, y1);
}
__device__ __forceinline__ float4 u_ld4(const IBArgs& a, const float2* p) {
    const float2* u = static_cast<const float2*>(a.u);
    if (!LBIB_CHK_ACCESS(a.diag, kSiteIbU, p, 16, u, u + a.plane))
        return make_float4(0.f, 0.f, 0.f, 0.f);
    return *reinterpret_cast<const float4*>(p);
}
template <typename V2>
__device__ __forceinline__ V2 u_ld(const IBArgs& a, const V2* p) {
    const V2* u = static_cast<const V2*>(a.u);
    if (!LBIB_CHK_ACCESS(a.diag, kSiteIbU, p, (int)sizeof(V2), u, u + a.plane)) {
        V2 z;
        z.x = 0;
        z.y = 0;
        return z;
    }
    return *p;
}

// Hookean spring of the edge A -> B with constant k and rest length L0: the
// force on A (B receives the opposite).  FP64 path: all FP64.  FP32 path: the
// stretch |d| - L0 = (|d|^2 - L0^2)/(|d| + L0) takes its cancelling difference
// in FP64 and the rest in FP32.
template <typename C>
__device__ __forceinline__ void spring(double2 A, double2 B, double L0, double kk, C* fx, C* fy) {
    const double dx = B.x - A.x, dy = B.y - A.y;
    if (sizeof(C) == 8) {
        const double len = sqrt(dx * dx + dy * dy);
        const double sc = kk * (len - L0) / len;
        *fx = (C)(sc * dx);
        *fy = (C)(sc * dy);
    } else {
        const double len2 = dx * dx + dy * dy;
        const float d2 = (float)(len2 - L0 * L0);
        const float len = sqrtf((float)len2);
        const float sc = (float)kk * (d2 / (len + (float)L0)) / len;
        *fx = (C)(sc * (float)dx);
        *fy = (C)(sc * (float)dy);
    }
}

// crossing abscissa of edge A -> B with row y, every operation rounded on its own
__device__ __forceinline__ double crossing_x(double2 A, double2 B, double yn) {
    return __dadd_rn(A.x, __ddiv_rn(__dmul_rn(__dsub_rn(yn, A.y), __dsub_rn(B.x, A.x)),
                                    __dsub_rn(B.y, A.y)));
}

// Mark in `mask` (1 bit per 4 consecutive nodes) the groups of the four
// support nodes of one kernel row: one atomicOr per 32-group word touched.
__device__ __forceinline__ void mark_row(const IBArgs& a, uint32_t* mask, int64_t rowbase,
                                         const int ix[4]) {
    if (!mask) return;
    int64_t wd = -1;
    uint32_t bits = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t g = (rowbase + ix[i]) >> 2;
        if ((g >> 5) != wd) {
            if (bits && LBIB_CHK_INDEX(a.diag, kSiteMask, wd, mask_words(a.plane)))
                atomicOr(mask + wd, bits);
            wd = g >> 5;
            bits = 0u;
        }
        bits |= 1u << (g & 31);
    }
    if (LBIB_CHK_INDEX(a.diag, kSiteMask, wd, mask_words(a.plane))) atomicOr(mask + wd, bits);
}

// OR `bits` into mask word `wd` through the CTA's table of the cell's words
// (open addressing in shared memory; the word goes to the mask once, at the
// flush after the spreading); a full table falls back to the global atomic.
__device__ __forceinline__ void mask_or_table(const IBArgs& a, uint32_t* mask, int64_t wd,
                                              uint32_t bits, uint32_t* mkey, uint32_t* mval) {
    if (!LBIB_CHK_INDEX(a.diag, kSiteMask, wd, mask_words(a.plane))) return;
    const uint32_t k = (uint32_t)wd;
    uint32_t h = (k * 2654435761u) >> (32 - kMaskTableLog2);
#pragma unroll 1
    for (int probe = 0; probe < 16; ++probe) {
        const uint32_t old = atomicCAS(mkey + h, kMaskEmpty, k);
        if (old == kMaskEmpty || old == k) {
            atomicOr(mval + h, bits);
            return;
        }
        h = (h + 1) & (uint32_t)(kMaskTable - 1);
    }
    atomicOr(mask + wd, bits);
}

// mark_row through the table
__device__ __forceinline__ void mark_row_table(const IBArgs& a, uint32_t* mask, int64_t rowbase,
                                               const int ix[4], uint32_t* mkey, uint32_t* mval) {
    if (!mask) return;
    int64_t wd = -1;
    uint32_t bits = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t g = (rowbase + ix[i]) >> 2;
        if ((g >> 5) != wd) {
            if (bits) mask_or_table(a, mask, wd, bits, mkey, mval);
            wd = g >> 5;
            bits = 0u;
        }
        bits |= 1u << (g & 31);
    }
    mask_or_table(a, mask, wd, bits, mkey, mval);
}

// Mark the groups of the nodes [s, e) of one row (no wrap inside the range)
// in `mask`: lanes take one 32-group word each.
__device__ __forceinline__ void mark_range(const IBArgs& a, uint32_t* mask, int64_t rowbase,
                                           int s, int e, int lane, int step = 32) {
    if (!mask || e <= s) return;
    const int64_t ga = (rowbase + s) >> 2, gb = (rowbase + e - 1) >> 2;
    for (int64_t w = (ga >> 5) + lane; w <= (gb >> 5); w += step) {
        const unsigned lo = (w == (ga >> 5)) ? (unsigned)(ga & 31) : 0u;
        const unsigned hi = (w == (gb >> 5)) ? (unsigned)(gb & 31) : 31u;
        const uint32_t bits = ((2u << hi) - 1u) & ~((1u << lo) - 1u);
        if (LBIB_CHK_INDEX(a.diag, kSiteMask, w, mask_words(a.plane))) atomicOr(mask + w, bits);
    }
}
// one node's group bit in a mask
__device__ __forceinline__ void mark_node(const IBArgs& a, uint32_t* mask, int64_t node) {
    const int64_t g = node >> 2;
    if (mask && LBIB_CHK_INDEX(a.diag, kSiteMask, g >> 5, mask_words(a.plane)))
        atomicOr(mask + (g >> 5), 1u << (g & 31));
}

// Labels of one cell (phase 3 of the IB kernels).  With scan_ok the per-row
// thresholds in thr/rowcnt are complete: one warp per row sorts them and
// fills each span [t_{2k}, t_{2k+1}) -- the nodes with an odd number of
// thresholds above them.  Otherwise every node of the box evaluates the
// crossing predicate over all edges in FP64 (the brute-force path).  Every
// inside node receives, with a.do_ids, the packed label (atomicMin: the lower
// cell index wins) and, when the cell has source bits, those bits in the
// source plane (atomicOr: a node inside several cells gets all their sources).
// OR the source bits into the source plane at one node
__device__ __forceinline__ void src_or_node(const IBArgs& a, int64_t node, uint32_t bits) {
    if (a.src_words) {
        uint32_t* w = static_cast<uint32_t*>(a.src) + node;
        if (LBIB_CHK_ACCESS(a.diag, kSiteIbLabel, w, 4, a.src,
                            static_cast<uint32_t*>(a.src) + a.plane))
            atomicOr(w, bits);
    } else {
        unsigned int* w = reinterpret_cast<unsigned int*>(static_cast<uint8_t*>(a.src) + (node & ~3ll));
        if (LBIB_CHK_ACCESS(a.diag, kSiteIbLabel, w, 4, a.src,
                            static_cast<uint8_t*>(a.src) + a.plane))
            atomicOr(w, bits << (8 * (int)(node & 3)));
    }
}

// OR the source bits into the bytes [s, e) of one row of the byte plane (row
// start 8-byte aligned): one 64-bit atomic per 8 nodes, lanes take words
__device__ __forceinline__ void src_or_range(const IBArgs& a, uint8_t* row, int s, int e,
                                             uint32_t bits, int lane, int step = 32) {
    if (e <= s) return;
    const unsigned long long rep = 0x0101010101010101ull * (unsigned long long)bits;
    unsigned long long* wrow = reinterpret_cast<unsigned long long*>(row);
    for (int w = (s >> 3) + lane; w <= ((e - 1) >> 3); w += step) {
        const int a0 = max(s - 8 * w, 0), a1 = min(e - 8 * w, 8);
        const unsigned long long m =
            (a1 - a0 == 8) ? ~0ull : (((1ull << (8 * (a1 - a0))) - 1ull) << (8 * a0));
        if (LBIB_CHK_ACCESS(a.diag, kSiteIbLabel, wrow + w, 8, a.src,
                            static_cast<uint8_t*>(a.src) + a.plane))
            atomicOr(wrow + w, rep & m);
    }
}

__device__ __forceinline__ void label_node(const IBArgs& a, int64_t node, uint32_t code,
                                           uint32_t bits) {
    if (a.do_ids && LBIB_CHK_ACCESS(a.diag, kSiteIbLabel, a.id + node, 4, a.id, a.id + a.plane))
        atomicMin(a.id + node, code);
    if (bits) src_or_node(a, node, bits);
}

static __device__ __forceinline__ void fill_labels_body(const IBArgs& a, int c, int n, const double2* sx,
                                         const int* rowcnt, int* thr, bool scan_ok, int I0,
                                         int J0, int rows, int cols, int tid, int nthreads) {
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthreads >> 5;
    // source bits go to the source plane only when the caller gave one
    const uint32_t cbits = (uint32_t)(a.srcf[c] & 0xF);
    const uint32_t bits = a.src ? cbits : 0u;
    const uint32_t code = ((uint32_t)c << 4) | cbits;
    const int wI0 = wrapi(I0, a.nx), wJ0 = wrapi(J0, a.ny);
    if (scan_ok && !a.do_ids && !a.src_words && a.src) {
        // source bits only (every step between outputs): one thread per row,
        // so all rows of the cell at once, each span a few 8-byte ORs
        for (int r = tid; r < rows; r += nthreads) {
            const int J = J0 + r;
            if (a.bc_y && (J < 0 || J >= a.ny)) continue;
            const int m = rowcnt[r];
            int* tr = thr + r * kMaxCross;
            for (int q = 1; q < m; ++q) {
                const int v = tr[q];
                int p = q - 1;
                while (p >= 0 && tr[p] > v) {
                    tr[p + 1] = tr[p];
                    --p;
                }
                tr[p + 1] = v;
            }
            int wJ = wJ0 + r;
            if (wJ >= a.ny) wJ -= a.ny;
            const int64_t rb = (int64_t)wJ * a.pitch;
            uint8_t* row = static_cast<uint8_t*>(a.src) + rb;
            if ((m & 1) == 0) {
                for (int k = 0; k + 1 < m; k += 2) {
                    const int lo = tr[k], hi = tr[k + 1];
                    if (hi <= lo) continue;
                    int ws = wI0 + (lo - I0);
                    if (ws >= a.nx) ws -= a.nx;
                    const int len = hi - lo;
                    const int e1 = ws + len <= a.nx ? ws + len : a.nx;
                    const int e2 = ws + len - a.nx;  // > 0 when the span wraps
                    src_or_range(a, row, ws, e1, bits, 0, 1);
                    mark_range(a, a.smask, rb, ws, e1, 0, 1);
                    if (e2 > 0) {
                        src_or_range(a, row, 0, e2, bits, 0, 1);
                        mark_range(a, a.smask, rb, 0, e2, 0, 1);
                    }
                }
            } else {  // odd count: the parity rule node by node
                for (int cc = 0; cc < cols; ++cc) {
                    const int I = I0 + cc;
                    int cnt = 0;
                    for (int q = 0; q < m; ++q) cnt += (tr[q] > I);
                    if (cnt & 1) {
                        int wI = wI0 + cc;
                        if (wI >= a.nx) wI -= a.nx;
                        label_node(a, rb + wI, code, bits);
                        mark_node(a, a.smask, rb + wI);
                    }
                }
            }
        }
        return;
    }
    if (scan_ok) {
        // one warp per row: sort the row's thresholds, then fill each span
        // [t_{2k}, t_{2k+1}) -- the nodes with an odd number of thresholds
        // above them
        for (int r = warp; r < rows; r += nwarps) {
            const int J = J0 + r;
            if (a.bc_y && (J < 0 || J >= a.ny)) continue;
            const int m = rowcnt[r];
            int* tr = thr + r * kMaxCross;
            if (lane == 0) {
                for (int q = 1; q < m; ++q) {
                    const int v = tr[q];
                    int p = q - 1;
                    while (p >= 0 && tr[p] > v) {
                        tr[p + 1] = tr[p];
                        --p;
                    }
                    tr[p + 1] = v;
                }
            }
            __syncwarp();
            int wJ = wJ0 + r;
            if (wJ >= a.ny) wJ -= a.ny;
            const int64_t rb = (int64_t)wJ * a.pitch;
            if ((m & 1) == 0) {
                for (int k = 0; k + 1 < m; k += 2) {
                    const int lo = tr[k], hi = tr[k + 1];
                    // byte plane: whole words per lane below; word plane: per node
                    const uint32_t nbits = a.src_words ? bits : 0u;
                    if (a.do_ids || nbits) {
                        for (int I = lo + lane; I < hi; I += 32) {
                            int wI = wI0 + (I - I0);
                            if (wI >= a.nx) wI -= a.nx;
                            label_node(a, rb + wI, code, nbits);
                        }
                    }
                    if (hi > lo) {  // the span's words and groups, split where it wraps
                        int ws = wI0 + (lo - I0);
                        if (ws >= a.nx) ws -= a.nx;
                        const int len = hi - lo;
                        const int e1 = ws + len <= a.nx ? ws + len : a.nx;
                        const int e2 = ws + len - a.nx;  // > 0 when the span wraps
                        if (a.do_ids) {
                            mark_range(a, a.lmask, rb, ws, e1, lane);
                            if (e2 > 0) mark_range(a, a.lmask, rb, 0, e2, lane);
                        }
                        if (bits) {
                            if (!a.src_words) {
                                uint8_t* row = static_cast<uint8_t*>(a.src) + rb;
                                src_or_range(a, row, ws, e1, bits, lane);
                                if (e2 > 0) src_or_range(a, row, 0, e2, bits, lane);
                            }
                            mark_range(a, a.smask, rb, ws, e1, lane);
                            if (e2 > 0) mark_range(a, a.smask, rb, 0, e2, lane);
                        }
                    }
                }
            } else {  // odd count: evaluate the parity rule node by node
                for (int cc = lane; cc < cols; cc += 32) {
                    const int I = I0 + cc;
                    int cnt = 0;
                    for (int q = 0; q < m; ++q) cnt += (tr[q] > I);
                    if (cnt & 1) {
                        int wI = wI0 + cc;
                        if (wI >= a.nx) wI -= a.nx;
                        label_node(a, rb + wI, code, bits);
                        if (a.do_ids) mark_node(a, a.lmask, rb + wI);
                        if (bits) mark_node(a, a.smask, rb + wI);
                    }
                }
            }
            __syncwarp();
        }
    } else {
        // brute force: the same predicate per node over all edges
        if (tid == 0) raise_flag(a.diag, kDiagRasterSlow);
        for (int e = tid; e < rows * cols; e += nthreads) {
            const int r = e / cols, cc = e % cols, J = J0 + r;
            if (a.bc_y && (J < 0 || J >= a.ny)) continue;
            const double xn = (double)(I0 + cc), yn = (double)J;
            bool inside = false;
            for (int t = 0; t < n; ++t) {
                const double2 A = sx[t], B = sx[(t == n - 1) ? 0 : t + 1];
                if ((A.y <= yn) != (B.y <= yn) && xn < crossing_x(A, B, yn)) inside = !inside;
            }
            if (inside) {
                int wI = wI0 + cc, wJ = wJ0 + r;
                if (wI >= a.nx) wI -= a.nx;
                if (wJ >= a.ny) wJ -= a.ny;
                const int64_t node = (int64_t)wJ * a.pitch + wI;
                label_node(a, node, code, bits);
                if (a.do_ids) mark_node(a, a.lmask, node);
                if (bits) mark_node(a, a.smask, node);
            }
        }
    }
}

// out of line: keeps the register budget of the callers that hold more state
// (the ensemble's persistent kernel)
static __device__ __noinline__ void fill_labels_call(const IBArgs& a, int c, int n,
                                                     const double2* sx, const int* rowcnt,
                                                     int* thr, bool scan_ok, int I0, int J0,
                                                     int rows, int cols, int tid, int nthreads) {
    fill_labels_body(a, c, n, sx, rowcnt, thr, scan_ok, I0, J0, rows, cols, tid, nthreads);
}

// Barrier of the NT threads that work on one cell: `bar` 0 with a CTA of NT
// threads, or a named barrier of its own for each NT-thread part of a larger
// CTA that works on several cells at once.
template <int NT>
__device__ __forceinline__ void cell_sync(int bar) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "n"(NT) : "memory");
}

// ---------------------------------------------------------------------------
// FP32 path.  GB300's FP64 rate is a small fraction of its FP32 rate, so the
// FP32 path keeps FP64 to what the storage rule and exactness need: each
// vertex position is FP64; per vertex and step it takes floor(X) and the
// fraction X - floor(X) once (FP64 -> int + float).  Everything else --
// kernel weights, edge vectors, springs, pressure, tension, scanline
// crossings -- is FP32 on (integer base, fraction) pairs:
//   * an edge vector is (base_b - base_a) + (frac_b - frac_a), accurate to
//     about 1e-7 LU whatever the coordinate magnitude;
//   * ceil(y) = base_y + (frac_y > 0) is exact, so the row predicate
//     (y_a <= J) != (y_b <= J) is evaluated exactly in integers;
//   * a crossing abscissa is computed in FP32 relative to its edge's first
//     vertex with an error bound E; if [x - E, x + E] holds no integer its
//     ceiling is the ceiling of the exact FP64 value, otherwise (rare) the
//     FP64 formula is evaluated, so labels stay identical to the FP64 rule.
// The (base, fraction) of X^{n+1} computed at the end of a launch is stored
// per vertex and reused by the interpolation of the next launch.

__device__ __forceinline__ void base_frac(double X, int* b, float* f) {
    const double fl = floor(X);
    *b = (int)fl;
    *f = (float)(X - fl);
}

__device__ __forceinline__ void weights_from_frac(float f, float w[4]) {
    float sn, cs;
    sincospif(0.5f * f, &sn, &cs);
    w[0] = 0.25f * (1.f - sn);
    w[1] = 0.25f * (1.f + cs);
    w[2] = 0.25f * (1.f + sn);
    w[3] = 0.25f * (1.f - cs);
}

__device__ __forceinline__ float2 edge_vec(int2 ba, float2 fa, int2 bb, float2 fb) {
    return make_float2((float)(bb.x - ba.x) + (fb.x - fa.x), (float)(bb.y - ba.y) + (fb.y - fa.y));
}

// spring force on the first vertex of an edge with vector d (FP32)
__device__ __forceinline__ float2 spring32(float2 d, float L0, float kk) {
    const float len2 = d.x * d.x + d.y * d.y;
    const float len = sqrtf(len2);
    const float sc = kk * ((len2 - L0 * L0) / (len + L0)) / len;
    return make_float2(sc * d.x, sc * d.y);
}

// The work of one cell by NT threads (thread index tid, barrier bar: the
// whole CTA, or one part of it).  Callers that run several cells through the
// same threads call it again for the next cell; the first barrier protects the
// shared arrays of the previous call.  GRIDDEP: the
// caller is a kernel of its own (programmatic launch after a lattice launch):
// the cell's constant data and its vertex state (written by the IB launch two
// launches back) are loaded through L2 before the wait, the u plane after it.
// INLINE_FILL: the label fill inlined (the 256-thread kernel: no spills, no
// parameter reads through a pointer; 1024^2 step 40.9 -> 38.4 us) or called
// out of line (the small-CTA kernels keep few registers, 18 CTAs of 64
// threads per SM, and the ensemble's persistent kernel its budget)
// OPTS = false compiles out the junction forces and mass sources (the
// ensemble has neither).  The force-mask bits go through the cell slot's
// table of mask words (one global OR per distinct word instead of one per
// vertex and stencil row: the small-CTA kernels of many cells, whose ORs to
// shared words throttle the launch; 4096^2, 9,801 cells: IB launch 104 -> 93
// us), or straight to the mask (the 256-thread kernel of few large cells,
// where the table's extra barrier lengthens each cell's chain: 1024^2, 400
// cells, 16.7 -> 22 us with it).
template <int NT, bool GRIDDEP, bool INLINE_FILL = true, bool OPTS = true,
          bool MASK_TABLE = (NT <= 128)>
static __device__ void ib_cell_f32(const IBArgs& a, int c, const IBShared32& S, int tid,
                                   int bar) {
    static_assert(NT % 64 == 0, "CTA size");
    constexpr int kIBThreads = NT;
    double2* sx = S.sx;
    int2* sb = S.sb;
    float2* sf = S.sf;
    int* rowcnt = S.rowcnt;
    int* thr = S.thr;
    int* sbox = S.sbox;
    int& s_flag = *S.s_flag;
    cell_sync<NT>(bar);

    const int v0 = __ldcg(a.off + c);
    const int n = __ldcg(a.off + c + 1) - v0;
    const int lane = tid & 31;
    // the checking build: the cell's vertices inside the vertex arrays
    const bool vok = LBIB_CHK_INDEX(a.diag, kSiteIbVertex, v0, (int64_t)__ldcg(a.off + a.n_cells)) &&
                     LBIB_CHK_INDEX(a.diag, kSiteIbVertex, (int64_t)v0 + n - 1,
                                    (int64_t)__ldcg(a.off + a.n_cells));
    if (n > S.maxv || n < 3 || !vok) {  // cannot happen for callers that size maxv from the cells
        if (GRIDDEP) {
            griddep_wait();
            griddep_launch_dependents();
        }
        if (tid == 0) raise_flag(a.diag, kDiagGeometry);
        return;
    }

    for (int r = tid; r < kMaxRows; r += NT) rowcnt[r] = 0;
    if (MASK_TABLE) {
        for (int i = tid; i < kMaskTable; i += NT) {
            S.mkey[i] = kMaskEmpty;
            S.mval[i] = 0u;
        }
    }
    if (tid == 0) {
        sbox[0] = INT_MAX; sbox[1] = INT_MIN; sbox[2] = INT_MAX; sbox[3] = INT_MIN;
        s_flag = 0;
    }

    // spring data of the vertices this thread will handle in phase 2, loaded
    // now so that phase 2 waits on no load: vertex tid (every thread: the whole
    // CTA computes forces when the cell is not labelled) and vertex tid + half
    // (the first half, which alone computes forces while the second half
    // scans the rows of a labelled cell)
    constexpr int half = kIBThreads / 2;
    float pL0[2] = {0.f, 0.f}, pk[2] = {0.f, 0.f}, pL0p[2] = {0.f, 0.f}, pkp[2] = {0.f, 0.f};
    float ppres = 0.f;
    if (a.do_prep && a.do_force) {
        ppres = (float)__ldcg(a.pres + c);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int t = tid + r * half;
            if (t < n && (r == 0 || tid < half)) {
                const int tp = (t == 0) ? n - 1 : t - 1;
                pL0[r] = (float)__ldcg(a.L0 + v0 + t);
                pk[r] = (float)__ldcg(a.k + v0 + t);
                pL0p[r] = (float)__ldcg(a.L0 + v0 + tp);
                pkp[r] = (float)__ldcg(a.k + v0 + tp);
            }
        }
    }
    // the vertex state of this thread's first vertex
    double2 X0 = make_double2(0.0, 0.0);
    int2 b0 = make_int2(0, 0);
    float2 f0 = make_float2(0.f, 0.f);
    if (tid < n) {
        X0 = __ldcg(a.xy + v0 + tid);
        if (a.do_move && a.vbase) {
            b0 = __ldcg(a.vbase + v0 + tid);
            f0 = __ldcg(a.vfrac + v0 + tid);
        }
    }
    if (GRIDDEP) {
        griddep_wait();
        griddep_launch_dependents();
    }

    // ---- (1) interpolate u^n at X^n and move; (base, frac) of the new X
    int ilo = INT_MAX, ihi = INT_MIN, jlo = INT_MAX, jhi = INT_MIN;
    bool finite = true;
    for (int t = tid; t < n; t += kIBThreads) {
        double2 X = (t == tid) ? X0 : a.xy[v0 + t];
        int2 b;
        float2 f;
        if (a.do_move) {
            if (a.vbase) {
                b = (t == tid) ? b0 : a.vbase[v0 + t];
                f = (t == tid) ? f0 : a.vfrac[v0 + t];
            } else {
                base_frac(X.x, &b.x, &f.x);
                base_frac(X.y, &b.y, &f.y);
            }
            float wx[4], wy[4];
            weights_from_frac(f.x, wx);
            weights_from_frac(f.y, wy);
            const float2* u = static_cast<const float2*>(a.u);
            float Ux = 0.f, Uy = 0.f;
            int ix[4];
            ix[0] = wrapi(b.x - 1, a.nx);
#pragma unroll
            for (int i = 1; i < 4; ++i) ix[i] = (ix[i - 1] + 1 == a.nx) ? 0 : ix[i - 1] + 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int J = b.y - 1 + j;
                if (a.bc_y) {
                    if (J < 0 || J >= a.ny) continue;
                } else {
                    J = wrapi(J, a.ny);
                }
                const float2* row = u + (int64_t)J * a.pitch;
                // the four nodes of the row, 16 bytes per load where aligned
                float2 v[4];
                if (ix[3] == ix[0] + 3) {
                    const float2* r0 = row + ix[0];
                    if ((ix[0] & 1) == 0) {
                        const float4 p0 = u_ld4(a, r0);
                        const float4 p1 = u_ld4(a, r0 + 2);
                        v[0] = make_float2(p0.x, p0.y);
                        v[1] = make_float2(p0.z, p0.w);
                        v[2] = make_float2(p1.x, p1.y);
                        v[3] = make_float2(p1.z, p1.w);
                    } else {
                        const float4 p1 = u_ld4(a, r0 + 1);
                        v[0] = u_ld(a, r0);
                        v[1] = make_float2(p1.x, p1.y);
                        v[2] = make_float2(p1.z, p1.w);
                        v[3] = u_ld(a, r0 + 3);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) v[i] = u_ld(a, row + ix[i]);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float w = wx[i] * wy[j];
                    Ux += v[i].x * w;
                    Uy += v[i].y * w;
                }
            }
            X.x += (double)Ux;
            X.y += (double)Uy;
            a.xy[v0 + t] = X;
        }
        base_frac(X.x, &b.x, &f.x);
        base_frac(X.y, &b.y, &f.y);
        sx[t] = X;
        sb[t] = b;
        sf[t] = f;
        if (a.do_prep && a.vbase) {
            a.vbase[v0 + t] = b;
            a.vfrac[v0 + t] = f;
        }
        finite = finite && isfinite(f.x) && isfinite(f.y) && b.x > -1000000000 &&
                 b.x < 1000000000 && b.y > -1000000000 && b.y < 1000000000;
        const int cyv = b.y + (f.y > 0.f ? 1 : 0);  // ceil(y), exact
        ilo = min(ilo, b.x);
        ihi = max(ihi, b.x);
        jlo = min(jlo, cyv);
        jhi = max(jhi, cyv);
    }
    if (!a.do_prep) return;
    ilo = __reduce_min_sync(0xffffffffu, ilo);
    ihi = __reduce_max_sync(0xffffffffu, ihi);
    jlo = __reduce_min_sync(0xffffffffu, jlo);
    jhi = __reduce_max_sync(0xffffffffu, jhi);
    finite = __all_sync(0xffffffffu, finite);
    cell_sync<NT>(bar);
    if (lane == 0) {
        atomicMin(&sbox[0], ilo);
        atomicMax(&sbox[1], ihi);
        atomicMin(&sbox[2], jlo);
        atomicMax(&sbox[3], jhi);
        if (!finite) s_flag = 2;
    }
    cell_sync<NT>(bar);
    if (OPTS && a.msrc_out && tid < 32) {
        // mass source of the cell (Sec. 3.2.3): S_c = rate + alpha (A0 - A_c),
        // A_c the shoelace area of the moved polygon about its first vertex
        const double a_c = cell_area_warp(sx, n, lane);
        if (lane == 0) static_cast<float*>(a.msrc_out)[c] = (float)mass_source(a, c, a_c);
    }
    // columns: floor(x) over the vertices, widened by one on each side (the
    // fractions are FP32); rows: every J with min ceil(y) <= J < max ceil(y),
    // exactly the rows some edge crosses
    const int I0 = sbox[0] - 1, I1 = sbox[1] + 1, J0 = sbox[2], J1 = sbox[3] - 1;
    // a box no wider than the lattice keeps the wrapped indices of the fill
    // within one period; anything wider means the geometry has blown up
    const bool geom_ok = s_flag == 0 && (I1 - I0) < a.nx && (J1 - J0) <= a.ny;
    if (a.do_mask && !geom_ok && tid == 0) raise_flag(a.diag, kDiagGeometry);
    // the cell is labelled when the caller wants the packed labels or the cell
    // has source bits to deposit
    const bool labels =
        a.do_mask && geom_ok && J1 >= J0 && (a.do_ids || (a.src && (a.srcf[c] & 0xF)));
    const int rows = J1 - J0 + 1, cols = I1 - I0 + 1;
    const bool scan = labels && rows <= kMaxRows;

    if (tid < half || !scan) {  // forces: the first half, or all threads without a scan
        if (a.do_force) {
            float2* force = static_cast<float2*>(a.force);
            const float p = ppres;
            const float ten = (float)a.tension;
            const int stride = scan ? half : kIBThreads;
            for (int t = tid, r = 0; t < n; t += stride, ++r) {
                const int tp = (t == 0) ? n - 1 : t - 1;
                const int tn = (t == n - 1) ? 0 : t + 1;
                const int2 b = sb[t];
                const float2 f = sf[t];
                const float2 dn = edge_vec(b, f, sb[tn], sf[tn]);   // X_{t+1} - X_t
                const float2 dp = edge_vec(sb[tp], sf[tp], b, f);   // X_t - X_{t-1}
                // prefetched for the first two vertices of this thread
                const bool pre1 = r == 1 && stride == half;  // tid + half, prefetched
                const float L0t = r == 0 ? pL0[0] : (pre1 ? pL0[1] : (float)a.L0[v0 + t]);
                const float kt = r == 0 ? pk[0] : (pre1 ? pk[1] : (float)a.k[v0 + t]);
                const float L0p = r == 0 ? pL0p[0] : (pre1 ? pL0p[1] : (float)a.L0[v0 + tp]);
                const float kp = r == 0 ? pkp[0] : (pre1 ? pkp[1] : (float)a.k[v0 + tp]);
                const float2 s0 = spring32(dn, L0t, kt);
                const float2 s1 = spring32(dp, L0p, kp);
                float Fx = s0.x - s1.x, Fy = s0.y - s1.y;
                // pressure p dA/dX: (p/2)(y_{t+1} - y_{t-1}, x_{t-1} - x_{t+1})
                Fx += 0.5f * p * (dn.y + dp.y);
                Fy -= 0.5f * p * (dn.x + dp.x);
                if (ten != 0.f) {  // Eq. membraneforce
                    const float ln = sqrtf(dn.x * dn.x + dn.y * dn.y);
                    const float lp = sqrtf(dp.x * dp.x + dp.y * dp.y);
                    Fx += ten * (dn.x / ln - dp.x / lp);
                    Fy += ten * (dn.y / ln - dp.y / lp);
                }
                if (OPTS && a.jpartner) {  // Eq. celljunctionforce (a launch without the move)
                    const float2 J = junction_force32(a, sx[t], a.jpartner[v0 + t]);
                    Fx += J.x;
                    Fy += J.y;
                }
                if (a.write_vforce) a.vforce[v0 + t] = make_double2((double)Fx, (double)Fy);

                float wx[4], wy[4];
                weights_from_frac(f.x, wx);
                weights_from_frac(f.y, wy);
                int ix[4];
                ix[0] = wrapi(b.x - 1, a.nx);
#pragma unroll
                for (int i = 1; i < 4; ++i) ix[i] = (ix[i - 1] + 1 == a.nx) ? 0 : ix[i - 1] + 1;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    int J = b.y - 1 + j;
                    if (a.bc_y) {
                        if (J < 0 || J >= a.ny) {
                            raise_flag(a.diag, kDiagWallStencil);
                            continue;
                        }
                    } else {
                        J = wrapi(J, a.ny);
                    }
                    float2* row = force + (int64_t)J * a.pitch;
                    float cx4[4], cy4[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float w = wx[i] * wy[j];
                        cx4[i] = Fx * w;
                        cy4[i] = Fy * w;
                    }
                    // the four nodes of the row: two 16-byte reductions when
                    // the row starts on an even node, 8 + 16 + 8 bytes when it
                    // starts on an odd one, one per node across the periodic seam
                    if (ix[3] == ix[0] + 3) {
                        float2* r0 = row + ix[0];
                        if ((ix[0] & 1) == 0) {
                            force_red2(a, r0, cx4[0], cy4[0], cx4[1], cy4[1]);
                            force_red2(a, r0 + 2, cx4[2], cy4[2], cx4[3], cy4[3]);
                        } else {
                            force_red1(a, r0, cx4[0], cy4[0]);
                            force_red2(a, r0 + 1, cx4[1], cy4[1], cx4[2], cy4[2]);
                            force_red1(a, r0 + 3, cx4[3], cy4[3]);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) spread_add(a, &row[ix[i]], cx4[i], cy4[i]);
                    }
                    if (MASK_TABLE)
                        mark_row_table(a, a.fmask, (int64_t)J * a.pitch, ix, S.mkey, S.mval);
                    else
                        mark_row(a, a.fmask, (int64_t)J * a.pitch, ix);
                }
            }
        }
    } else if (scan) {
        for (int e = tid - half; e < n; e += half) {
            const int eb = (e == n - 1) ? 0 : e + 1;
            const int2 ba = sb[e], bb = sb[eb];
            const float2 fa = sf[e], fb = sf[eb];
            const int cya = ba.y + (fa.y > 0.f ? 1 : 0), cyb = bb.y + (fb.y > 0.f ? 1 : 0);
            if (cya == cyb) continue;
            // rows J with (y_a <= J) != (y_b <= J): min(cy) <= J < max(cy)
            const int jl = min(cya, cyb), jh = max(cya, cyb) - 1;
            const float2 d = edge_vec(ba, fa, bb, fb);
            const float ratio = fabsf(d.x) / fabsf(d.y);
            for (int J = jl; J <= jh; ++J) {
                // x_c - base_a.x = frac_a.x + (J - y_a)(x_b - x_a)/(y_b - y_a)
                const float pr = (float)(J - ba.y) - fa.y;
                const float xr = fa.x + (pr * d.x) / d.y;
                const float E = 9.5367431640625e-07f * (4.f + 4.f * ratio + fabsf(d.x) + fabsf(xr));
                const float clo = ceilf(xr - E), chi = ceilf(xr + E);
                int ti;
                if (clo == chi) {
                    ti = ba.x + (int)clo;
                } else {
                    const double tc = ceil(crossing_x(sx[e], sx[eb], (double)J));
                    ti = tc < (double)I0 ? I0 : (tc > (double)(I1 + 1) ? I1 + 1 : (int)tc);
                }
                ti = ti < I0 ? I0 : (ti > I1 + 1 ? I1 + 1 : ti);
                const int slot = atomicAdd(&rowcnt[J - J0], 1);
                if (slot < kMaxCross)
                    thr[(J - J0) * kMaxCross + slot] = ti;
                else
                    s_flag = 1;
            }
        }
    }
    // every distinct force-mask word of the cell into the mask, once
    if (MASK_TABLE && a.do_force && a.fmask) {
        cell_sync<NT>(bar);
        for (int i = tid; i < kMaskTable; i += NT) {
            const uint32_t k = S.mkey[i];
            if (k != kMaskEmpty) atomicOr(a.fmask + k, S.mval[i]);
        }
    }
    if (!labels) return;  // uniform over the CTA
    cell_sync<NT>(bar);
    if (INLINE_FILL)
        fill_labels_body(a, c, n, sx, rowcnt, thr, scan && s_flag == 0, I0, J0, rows, cols, tid,
                         NT);
    else
        fill_labels_call(a, c, n, sx, rowcnt, thr, scan && s_flag == 0, I0, J0, rows, cols, tid,
                         NT);
}

}  // namespace lbib
