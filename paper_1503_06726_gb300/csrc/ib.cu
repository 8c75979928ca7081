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
#include <type_traits>

#include "lbib_internal.cuh"

namespace lbib {

__device__ __forceinline__ int wrapi(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ double delta1d(double r) {
    double a = fabs(r);
    return a > 2.0 ? 0.0 : 0.25 * (1.0 + cospi(0.5 * a));
}
__device__ __forceinline__ float delta1d(float r) {
    float a = fabsf(r);
    return a > 2.f ? 0.f : 0.25f * (1.f + cospif(0.5f * a));
}

// weights of the 4 support nodes along one axis, base = floor(X) - 1
template <typename C>
__device__ __forceinline__ void axis_weights(double X, int* base, C w[4]) {
    double fl = floor(X);
    *base = (int)fl - 1;
    if (sizeof(C) == 8) {
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = (C)delta1d((fl - 1.0 + a) - X);
    } else {
        float fr = (float)(X - fl);  // in [0, 1), exact in double
#pragma unroll
        for (int a = 0; a < 4; ++a) w[a] = (C)delta1d((float)(a - 1) - fr);
    }
}

// spread one weighted force into a node: FP32 uses the float2 vector atomic
__device__ __forceinline__ void spread_add(float2* p, float fx, float fy) {
    atomicAdd(p, make_float2(fx, fy));
}
__device__ __forceinline__ void spread_add(double2* p, double fx, double fy) {
    atomicAdd(&p->x, fx);
    atomicAdd(&p->y, fy);
}

__device__ __forceinline__ double dmin(double a, double b) { return a < b ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

template <typename C>
__global__ void __launch_bounds__(128) ib_cell_kernel(IBArgs a) {
    using V2 = typename std::conditional<sizeof(C) == 8, double2, float2>::type;
    __shared__ double2 sx[kMaxVertsPerCell];
    __shared__ V2 sedge[kMaxVertsPerCell];
    __shared__ int rowcnt[kMaxRows];
    __shared__ int thr[kMaxRows * kMaxCross];
    __shared__ double red[4][4];
    __shared__ int s_overflow;

    const int c = blockIdx.x;
    const int v0 = a.off[c];
    const int n = a.off[c + 1] - v0;
    const int tid = threadIdx.x;

    // ---- (1) interpolate and move, or just load
    for (int t = tid; t < n; t += blockDim.x) {
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
                    V2 v = row[ix[i]];
                    C w = wx[i] * wy[j];
                    Ux += v.x * w;
                    Uy += v.y * w;
                }
            }
            X.x += (double)Ux;
            X.y += (double)Uy;
            a.xy[v0 + t] = X;
        }
        sx[t] = X;
    }
    if (!a.do_prep) return;
    __syncthreads();

    // ---- (2) vertex forces and spreading
    // spring of edge t -> t+1, once per edge: the force on vertex t (its
    // partner t+1 receives the opposite).  FP64 path: all FP64.  FP32 path:
    // the stretch |d| - L0 = (|d|^2 - L0^2)/(|d| + L0) takes its cancelling
    // difference in FP64 and the rest in FP32.
    for (int t = tid; t < n; t += blockDim.x) {
        const double2 X = sx[t], Xn = sx[(t == n - 1) ? 0 : t + 1];
        const double dx = Xn.x - X.x, dy = Xn.y - X.y;
        const double L0 = a.L0[v0 + t], kk = a.k[v0 + t];
        V2 sp;
        if (sizeof(C) == 8) {
            double len = sqrt(dx * dx + dy * dy);
            double sc = kk * (len - L0) / len;
            sp.x = (C)(sc * dx);
            sp.y = (C)(sc * dy);
        } else {
            const double len2 = dx * dx + dy * dy;
            const float d2 = (float)(len2 - L0 * L0);
            const float len = sqrtf((float)len2);
            const float sc = (float)kk * (d2 / (len + (float)L0)) / len;
            sp.x = (C)(sc * (float)dx);
            sp.y = (C)(sc * (float)dy);
        }
        sedge[t] = sp;
    }
    __syncthreads();
    {
        V2* force = static_cast<V2*>(a.force);
        const C p = (C)a.pres[c];
        const C ten = (C)a.tension;
        for (int t = tid; t < n; t += blockDim.x) {
            const int tp = (t == 0) ? n - 1 : t - 1;
            const int tn = (t == n - 1) ? 0 : t + 1;
            const double2 X = sx[t], Xp = sx[tp], Xn = sx[tn];
            const V2 e0 = sedge[t], e1 = sedge[tp];
            C Fx = e0.x - e1.x, Fy = e0.y - e1.y;
            // pressure p dA/dX for a CCW polygon
            Fx += C(0.5) * p * (C)(Xn.y - Xp.y);
            Fy += C(0.5) * p * (C)(Xp.x - Xn.x);
            if (ten != C(0)) {  // Eq. membraneforce
                const C ax = (C)(Xp.x - X.x), ay = (C)(Xp.y - X.y);
                const C bx = (C)(Xn.x - X.x), by = (C)(Xn.y - X.y);
                const C la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
                Fx += ten * (ax / la + bx / lb);
                Fy += ten * (ay / la + by / lb);
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
                        atomicOr(a.diag + kDiagWallStencil, 1u);
                        continue;
                    }
                } else {
                    J = wrapi(J, a.ny);
                }
                V2* row = force + (int64_t)J * a.pitch;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const C w = wx[i] * wy[j];
                    spread_add(&row[ix[i]], Fx * w, Fy * w);
                }
            }
        }
    }

    if (!a.do_mask) return;

    // ---- (3) labels: bounding box
    double xmn = 1e300, xmx = -1e300, ymn = 1e300, ymx = -1e300;
    for (int t = tid; t < n; t += blockDim.x) {
        double2 X = sx[t];
        xmn = dmin(xmn, X.x); xmx = dmax(xmx, X.x);
        ymn = dmin(ymn, X.y); ymx = dmax(ymx, X.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xmn = dmin(xmn, __shfl_xor_sync(0xffffffffu, xmn, o));
        xmx = dmax(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
        ymn = dmin(ymn, __shfl_xor_sync(0xffffffffu, ymn, o));
        ymx = dmax(ymx, __shfl_xor_sync(0xffffffffu, ymx, o));
    }
    const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    if (lane == 0) {
        red[0][warp] = xmn; red[1][warp] = xmx; red[2][warp] = ymn; red[3][warp] = ymx;
    }
    if (tid == 0) s_overflow = 0;
    __syncthreads();
    xmn = red[0][0]; xmx = red[1][0]; ymn = red[2][0]; ymx = red[3][0];
    for (int w = 1; w < nwarps; ++w) {
        xmn = dmin(xmn, red[0][w]); xmx = dmax(xmx, red[1][w]);
        ymn = dmin(ymn, red[2][w]); ymx = dmax(ymx, red[3][w]);
    }
    // A bounding box that is not finite or wider than the lattice means the
    // geometry has blown up: flag it and leave the labels empty, so that the
    // loops below stay bounded by the lattice size.
    if (!(isfinite(xmn) && isfinite(xmx) && isfinite(ymn) && isfinite(ymx)) ||
        xmx - xmn > (double)a.nx || ymx - ymn > (double)a.ny || fabs(xmn) > 1e9 ||
        fabs(ymn) > 1e9) {
        if (tid == 0) atomicOr(a.diag + kDiagGeometry, 1u);
        return;
    }
    const int I0 = (int)floor(xmn), I1 = (int)ceil(xmx);
    const int J0 = (int)floor(ymn), J1 = (int)ceil(ymx);
    const int rows = J1 - J0 + 1, cols = I1 - I0 + 1;
    const uint32_t code = ((uint32_t)c << 4) | (uint32_t)(a.srcf[c] & 0xF);

    bool scan = rows <= kMaxRows;
    if (scan) {
        for (int r = tid; r < rows; r += blockDim.x) rowcnt[r] = 0;
        __syncthreads();
        for (int t = tid; t < n; t += blockDim.x) {
            const double2 A = sx[t], B = sx[(t == n - 1) ? 0 : t + 1];
            const double lo = dmin(A.y, B.y), hi = dmax(A.y, B.y);
            int jlo = (int)ceil(lo) - 1, jhi = (int)ceil(hi);
            if (jlo < J0) jlo = J0;
            if (jhi > J1) jhi = J1;
            for (int J = jlo; J <= jhi; ++J) {
                const double yn = (double)J;
                if ((A.y <= yn) != (B.y <= yn)) {
                    // x_c = x_a + (y - y_a)(x_b - x_a)/(y_b - y_a), each operation rounded
                    double xc = __dadd_rn(
                        A.x, __ddiv_rn(__dmul_rn(__dsub_rn(yn, A.y), __dsub_rn(B.x, A.x)),
                                       __dsub_rn(B.y, A.y)));
                    double tc = ceil(xc);
                    int ti = tc < (double)I0 ? I0 : (tc > (double)(I1 + 1) ? I1 + 1 : (int)tc);
                    int slot = atomicAdd(&rowcnt[J - J0], 1);
                    if (slot < kMaxCross)
                        thr[(J - J0) * kMaxCross + slot] = ti;
                    else
                        s_overflow = 1;
                }
            }
        }
        __syncthreads();
        scan = (s_overflow == 0);
    }
    uint32_t* id = a.id;
    if (scan) {
        // node e of the box = (row r, column cc), advanced by blockDim.x each
        // iteration without divisions; wrapped indices follow incrementally
        const int step_r = blockDim.x / cols, step_c = blockDim.x % cols;
        int r = tid / cols, cc = tid % cols;
        const int wI0 = wrapi(I0, a.nx), wJ0 = wrapi(J0, a.ny);
        for (; r < rows; r += step_r, cc += step_c) {
            if (cc >= cols) {
                cc -= cols;
                ++r;
                if (r >= rows) break;
            }
            const int J = J0 + r, I = I0 + cc;
            if (a.bc_y && (J < 0 || J >= a.ny)) continue;
            const int m = rowcnt[r];
            int cnt = 0;
            for (int q = 0; q < m; ++q) cnt += (thr[r * kMaxCross + q] > I);
            if (cnt & 1) {
                int wI = wI0 + cc, wJ = wJ0 + r;
                if (wI >= a.nx) wI -= a.nx;
                if (wJ >= a.ny) wJ -= a.ny;
                atomicMin(id + (int64_t)wJ * a.pitch + wI, code);
            }
        }
    } else {
        // brute force: the same predicate per node over all edges
        if (tid == 0) atomicAdd(a.diag + kDiagRasterSlow, 1u);
        for (int e = tid; e < rows * cols; e += blockDim.x) {
            const int r = e / cols, I = I0 + e % cols, J = J0 + r;
            if (a.bc_y && (J < 0 || J >= a.ny)) continue;
            const double xn = (double)I, yn = (double)J;
            bool inside = false;
            for (int t = 0; t < n; ++t) {
                const double2 A = sx[t], B = sx[(t == n - 1) ? 0 : t + 1];
                if ((A.y <= yn) != (B.y <= yn)) {
                    double xc = __dadd_rn(
                        A.x, __ddiv_rn(__dmul_rn(__dsub_rn(yn, A.y), __dsub_rn(B.x, A.x)),
                                       __dsub_rn(B.y, A.y)));
                    if (xn < xc) inside = !inside;
                }
            }
            if (inside) atomicMin(id + (int64_t)wrapi(J, a.ny) * a.pitch + wrapi(I, a.nx), code);
        }
    }
}

cudaError_t launch_ib(int precision, const IBArgs& a, cudaStream_t s) {
    if (a.n_cells <= 0) return cudaSuccess;
    if (precision == LBIB_FP64)
        ib_cell_kernel<double><<<a.n_cells, 128, 0, s>>>(a);
    else
        ib_cell_kernel<float><<<a.n_cells, 128, 0, s>>>(a);
    return cudaGetLastError();
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
