// ib.cu -- immersed-boundary side of the coupled step, one CTA per cell.
//
// A cell's vertices live in shared memory for the whole CTA, so the chain
//   interpolate u^n at X^n -> X^{n+1} = X^n + U^n      (Eq. conversion2, Fig. 1)
//   label the lattice nodes inside the new polygon      (Fig. 2, domainID)
//   vertex forces from springs, pressure, tension       (Sec. 3.2.3)
//   spread the forces to the 4x4 kernel support        (Eq. forcedistribution)
// runs in one launch between two lattice updates; no grid-wide sync is needed
// because every step only needs the cell's own vertices.
//
// Kernel of Eq. 1Dkernel: delta1D(r) = (1 + cos(pi r / 2)) / 4 for |r| <= 2,
// the 2-D kernel is delta1D(dx) delta1D(dy) over nodes floor(X)-1 .. floor(X)+2.
//
// Labelling: a node is inside a polygon by the crossing-number rule, half-open
// in y: edge a->b crosses row y when (y_a <= y) != (y_b <= y) and counts when
// x < x_a + (y - y_a)(x_b - x_a)/(y_b - y_a).  The CTA evaluates that crossing
// abscissa once per (edge, row) -- a scanline -- and keeps, per row, the
// integer thresholds ceil(x_c): a node at integer x is inside iff an odd
// number of thresholds exceed it.  This is the same predicate node by node,
// evaluated with explicitly rounded FP64 operations (no contraction), so the
// labels are exact.  Overlapping cells: the lowest cell index wins (atomicMin
// on the packed label cell << 4 | source bits).
#include <climits>
#include <type_traits>

#include "ib_cell.cuh"

namespace lbib {

template <typename C>
__global__ void __launch_bounds__(kIBThreads) ib_cell_kernel(IBArgs a) {
    using V2 = typename std::conditional<sizeof(C) == 8, double2, float2>::type;
    __shared__ double2 sx[kMaxVertsPerCell];
    __shared__ int rowcnt[kMaxRows];
    __shared__ int thr[kMaxRows * kMaxCross];
    __shared__ int sbox[4];  // I0, I1, J0, J1
    __shared__ int s_flag;   // 1: a scanline row overflowed, 2: geometry not finite

    const int c = blockIdx.x;
    const int v0 = __ldcg(a.off + c);
    const int n = __ldcg(a.off + c + 1) - v0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = kIBThreads / 32;
    // everything below reads the u plane of the lattice launch just before
    // (programmatic launch) or writes what it reads
    griddep_wait();
    griddep_launch_dependents();
    // the shared arrays hold kMaxVertsPerCell vertices and a polygon needs
    // three; callers that pass device offsets unchecked (the allocation-free
    // step) get the geometry flag instead of an access past sx
    const bool vok = LBIB_CHK_INDEX(a.diag, kSiteIbVertex, v0, (int64_t)__ldcg(a.off + a.n_cells)) &&
                     LBIB_CHK_INDEX(a.diag, kSiteIbVertex, (int64_t)v0 + n - 1,
                                    (int64_t)__ldcg(a.off + a.n_cells));
    if (n > kMaxVertsPerCell || n < 3 || !vok) {
        if (tid == 0) raise_flag(a.diag, kDiagGeometry);
        return;
    }

    if (tid < kMaxRows) rowcnt[tid] = 0;
    if (tid == 0) {
        sbox[0] = INT_MAX; sbox[1] = INT_MIN; sbox[2] = INT_MAX; sbox[3] = INT_MIN;
        s_flag = 0;
    }

    // ---- (1) interpolate u^n at X^n and move (or just load); integer bounding box
    int ilo = INT_MAX, ihi = INT_MIN, jlo = INT_MAX, jhi = INT_MIN;
    bool finite = true;
    for (int t = tid; t < n; t += kIBThreads) {
        double2 X = a.xy[v0 + t];
        if (a.do_move) {
            int bx, by;
            C wx[4], wy[4];
            axis_weights<C>(X.x, &bx, wx);
            axis_weights<C>(X.y, &by, wy);
            const V2* u = static_cast<const V2*>(a.u);
            C Ux = C(0), Uy = C(0);
            int ix[4];
            ix[0] = wrapi(bx, a.nx);
#pragma unroll
            for (int i = 1; i < 4; ++i) ix[i] = (ix[i - 1] + 1 == a.nx) ? 0 : ix[i - 1] + 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int J = by + j;
                if (a.bc_y) {
                    if (J < 0 || J >= a.ny) continue;
                } else {
                    J = wrapi(J, a.ny);
                }
                const V2* row = u + (int64_t)J * a.pitch;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const V2 v = u_ld(a, row + ix[i]);
                    const C w = wx[i] * wy[j];
                    Ux += v.x * w;
                    Uy += v.y * w;
                }
            }
            X.x += (double)Ux;
            X.y += (double)Uy;
            a.xy[v0 + t] = X;
        }
        sx[t] = X;
        finite = finite && isfinite(X.x) && isfinite(X.y) && fabs(X.x) < 1e9 && fabs(X.y) < 1e9;
        ilo = min(ilo, __double2int_rd(X.x));
        ihi = max(ihi, __double2int_ru(X.x));
        jlo = min(jlo, __double2int_rd(X.y));
        jhi = max(jhi, __double2int_ru(X.y));
    }
    if (!a.do_prep) return;
    ilo = __reduce_min_sync(0xffffffffu, ilo);
    ihi = __reduce_max_sync(0xffffffffu, ihi);
    jlo = __reduce_min_sync(0xffffffffu, jlo);
    jhi = __reduce_max_sync(0xffffffffu, jhi);
    finite = __all_sync(0xffffffffu, finite);
    __syncthreads();  // sbox / rowcnt initialised
    if (lane == 0) {
        atomicMin(&sbox[0], ilo);
        atomicMax(&sbox[1], ihi);
        atomicMin(&sbox[2], jlo);
        atomicMax(&sbox[3], jhi);
        if (!finite) s_flag = 2;
    }
    __syncthreads();
    if (a.msrc_out && warp == 0) {  // the cell's mass source (Sec. 3.2.3)
        const double a_c = cell_area_warp(sx, n, lane);
        if (lane == 0) static_cast<C*>(a.msrc_out)[c] = (C)mass_source(a, c, a_c);
    }
    const int I0 = sbox[0], I1 = sbox[1], J0 = sbox[2], J1 = sbox[3];
    // Labels need a finite box no wider than the lattice; otherwise the
    // geometry has blown up: flag it and leave the labels empty so that every
    // loop below stays bounded by the lattice size.
    const bool geom_ok = s_flag == 0 && (I1 - I0) <= a.nx && (J1 - J0) <= a.ny;
    if (a.do_mask && !geom_ok && tid == 0) raise_flag(a.diag, kDiagGeometry);
    // the cell is labelled when the caller wants the packed labels or the cell
    // has source bits to deposit
    const bool labels = a.do_mask && geom_ok && (a.do_ids || (a.src && (a.srcf[c] & 0xF)));
    const int rows = J1 - J0 + 1, cols = I1 - I0 + 1;
    const bool scan = labels && rows <= kMaxRows;

    // ---- (2) first half of the CTA: vertex forces and spreading;
    //          second half: scanline crossings of every edge
    constexpr int half = kIBThreads / 2;
    if (tid < half) {
      if (a.do_force) {
        V2* force = static_cast<V2*>(a.force);
        const C p = (C)a.pres[c];
        const C ten = (C)a.tension;
        for (int t = tid; t < n; t += half) {
            const int tp = (t == 0) ? n - 1 : t - 1;
            const int tn = (t == n - 1) ? 0 : t + 1;
            const double2 X = sx[t], Xp = sx[tp], Xn = sx[tn];
            C ax_, ay_, bx_, by_;
            spring<C>(X, Xn, a.L0[v0 + t], a.k[v0 + t], &ax_, &ay_);
            spring<C>(Xp, X, a.L0[v0 + tp], a.k[v0 + tp], &bx_, &by_);
            C Fx = ax_ - bx_, Fy = ay_ - by_;
            // pressure p dA/dX for a CCW polygon
            Fx += C(0.5) * p * (C)(Xn.y - Xp.y);
            Fy += C(0.5) * p * (C)(Xp.x - Xn.x);
            if (ten != C(0)) {  // Eq. membraneforce
                const C ux_ = (C)(Xp.x - X.x), uy_ = (C)(Xp.y - X.y);
                const C vx_ = (C)(Xn.x - X.x), vy_ = (C)(Xn.y - X.y);
                const C la = sqrt(ux_ * ux_ + uy_ * uy_), lb = sqrt(vx_ * vx_ + vy_ * vy_);
                Fx += ten * (ux_ / la + vx_ / lb);
                Fy += ten * (uy_ / la + vy_ / lb);
            }
            if (a.jpartner) {  // Eq. celljunctionforce (a launch without the move)
                const double2 J = junction_force64(a, X, a.jpartner[v0 + t]);
                Fx += (C)J.x;
                Fy += (C)J.y;
            }
            if (a.write_vforce) a.vforce[v0 + t] = make_double2((double)Fx, (double)Fy);

            int bxi, byi;
            C wx[4], wy[4];
            axis_weights<C>(X.x, &bxi, wx);
            axis_weights<C>(X.y, &byi, wy);
            int ix[4];
            ix[0] = wrapi(bxi, a.nx);
#pragma unroll
            for (int i = 1; i < 4; ++i) ix[i] = (ix[i - 1] + 1 == a.nx) ? 0 : ix[i - 1] + 1;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int J = byi + j;
                if (a.bc_y) {
                    if (J < 0 || J >= a.ny) {
                        raise_flag(a.diag, kDiagWallStencil);
                        continue;
                    }
                } else {
                    J = wrapi(J, a.ny);
                }
                V2* row = force + (int64_t)J * a.pitch;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const C w = wx[i] * wy[j];
                    spread_add(a, &row[ix[i]], Fx * w, Fy * w);
                }
                mark_row(a, a.fmask, (int64_t)J * a.pitch, ix);
            }
        }
      }
    } else if (scan) {
        for (int e = tid - half; e < n; e += half) {
            const double2 A = sx[e], B = sx[(e == n - 1) ? 0 : e + 1];
            const double lo = fmin(A.y, B.y), hi = fmax(A.y, B.y);
            int jl = __double2int_ru(lo) - 1, jh = __double2int_ru(hi);
            if (jl < J0) jl = J0;
            if (jh > J1) jh = J1;
            for (int J = jl; J <= jh; ++J) {
                const double yn = (double)J;
                if ((A.y <= yn) != (B.y <= yn)) {
                    const double tc = ceil(crossing_x(A, B, yn));
                    const int ti = tc < (double)I0 ? I0 : (tc > (double)(I1 + 1) ? I1 + 1 : (int)tc);
                    const int slot = atomicAdd(&rowcnt[J - J0], 1);
                    if (slot < kMaxCross)
                        thr[(J - J0) * kMaxCross + slot] = ti;
                    else
                        s_flag = 1;
                }
            }
        }
    }
    if (!labels) return;  // uniform over the CTA
    __syncthreads();

    fill_labels_call(a, c, n, sx, rowcnt, thr, scan && s_flag == 0, I0, J0, rows, cols, threadIdx.x,
                kIBThreads);
}


// FP32 path: dynamic shared memory sized for the largest cell, NT threads
template <int NT>
__device__ __forceinline__ void ib_f32_body(const IBArgs& a, int maxv) {
    extern __shared__ __align__(16) unsigned char ib_smem[];
    const IBShared32 S = ib_shared32_view(ib_smem, maxv);
    ib_cell_f32<NT, true, NT == 256>(a, blockIdx.x, S, threadIdx.x, 0);
}

// the 128- and 256-thread kernels at the registers the compiler chooses
template <int NT>
__global__ void __launch_bounds__(NT) ib_cell_kernel_f32(IBArgs a, int maxv) {
    ib_f32_body<NT>(a, maxv);
}

// the 64-thread kernel (many small cells) held to 56 registers, 18 CTAs per
// SM instead of 16 at its natural 64: more cells in flight for a
// latency-bound launch (C3, 9,801 cells: 107.7 -> 104.6 us)
__global__ void __launch_bounds__(64, 18) ib_cell_kernel_f32_64(IBArgs a, int maxv) {
    ib_f32_body<64>(a, maxv);
}

cudaError_t launch_ib(int precision, const IBArgs& a, int maxv_cell, cudaStream_t s, bool pdl) {
    if (a.n_cells <= 0) return cudaSuccess;
    if (precision == LBIB_FP64)
        return launch_kernel(ib_cell_kernel<double>, dim3(a.n_cells), dim3(kIBThreads), 0, s, pdl,
                             a);
    // small, numerous cells: 128-thread CTAs and shared memory sized to the
    // largest cell let many more CTAs be resident per SM
    int maxv = maxv_cell < 3 ? 3 : (maxv_cell > kMaxVertsPerCell ? kMaxVertsPerCell : maxv_cell);
    maxv = (maxv + 7) / 8 * 8;
    const size_t smem = kIBSmemFixed + (size_t)maxv * kIBSmemPerVertex;
    if (maxv <= 64 && a.n_cells >= 2048)
        return launch_kernel(ib_cell_kernel_f32_64, dim3(a.n_cells), dim3(64), smem, s, pdl, a,
                             maxv);
    if (maxv <= 128 && a.n_cells >= 2048)
        return launch_kernel(ib_cell_kernel_f32<128>, dim3(a.n_cells), dim3(128), smem, s, pdl, a,
                             maxv);
    return launch_kernel(ib_cell_kernel_f32<256>, dim3(a.n_cells), dim3(256), smem, s, pdl, a,
                         maxv);
}

// Per-cell shoelace area relative to the first vertex, FP64 (computeAreas).
__global__ void areas_kernel(const double2* xy, const int32_t* off, int n_cells, double* area) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n_cells) return;
    const int v0 = off[c], n = off[c + 1] - v0;
    const double2 P0 = xy[v0];
    double s = 0.0;
    for (int t = lane; t < n; t += 32) {
        double2 A = xy[v0 + t], B = xy[v0 + ((t == n - 1) ? 0 : t + 1)];
        double xl = A.x - P0.x, yl = A.y - P0.y, xm = B.x - P0.x, ym = B.y - P0.y;
        s += xl * ym - xm * yl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) area[c] = 0.5 * s;
}

cudaError_t launch_areas(const double2* xy, const int32_t* off, int n_cells, double* area,
                         cudaStream_t s) {
    if (n_cells <= 0) return cudaSuccess;
    areas_kernel<<<(n_cells + 3) / 4, 128, 0, s>>>(xy, off, n_cells, area);
    return cudaGetLastError();
}

}  // namespace lbib
