/*
 * lbib_oracle.c -- plain, slow FP64 CPU oracle of the LBIBCell coupled step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path never calls, links or includes anything here, and this file shares no
 * code, header, table or constant generator with it.
 *
 * Every routine follows one passage of Tanaka, Sichau & Iber,
 * "LBIBCell: a cell-based simulation environment for morphogenetic problems"
 * (arXiv:1503.06726), written as directly as possible: naive loops over nodes
 * and directions, a full copy for streaming, serial spreading in vertex order.
 * Where the paper is silent or garbled the reading taken is stated beside the
 * code.  Build: gcc -O2 -ffp-contract=off (no FMA contraction, so that the
 * point-in-polygon decisions are taken in plain IEEE double everywhere).
 *
 * Lattice conventions: node (i,j) at position (i,j), linear index j*nx+i.
 * Populations are stored as post-collision values f*_q(x) in planes q*N + idx;
 * a step first streams (pulls) them, then collides.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny, bc_y;      /* bc_y: 0 periodic, 1 half-way bounce-back walls at y=-1/2, ny-1/2 */
    int32_t n_species;
    double tau, rho0;
    double D[4], decay[4], react[4][4], src_rate[4];
    int32_t forcing;           /* 0 Guo et al. 2002, 1 the paper's simple term (Eq. bgkequation) */
    int32_t react_model;       /* 0 linear (react, decay); 1 Schnakenberg on species 0 and 1 */
    int32_t noflux;            /* bit s: species s is confined to its domain (no-flux membranes) */
    int32_t noflux_scheme;     /* 0: the equilibrium closure of Sec. 6.1; 1: half-way bounce-back */
    double schnak[3];          /* gamma, a, b of the Schnakenberg reaction */
    double junction_k, junction_l0, junction_lmax;   /* Eq. celljunctionforce */
    int32_t junction_period;   /* renew the junctions every this many steps (0 = none) */
    int32_t pad2;
    double mass_alpha;         /* gain of the cell area controller (Sec. 3.2.3) */
    double pressure_rho;       /* density prescribed at internal pressure nodes */
    double mass_beta;          /* mass source beta phi_s inside cells (reading c32) */
    int32_t mass_species;      /* the species s of that source */
    int32_t noflux_dynamic;    /* confined species follow the cells' labels of each step */
} orc_params;

/* D2Q9 velocities: v0 = 0; v1..v4 = (cos, sin)(pi(i-1)/2); v5..v8 the diagonals
 * sqrt(2)(cos, sin)(pi(i-1)/2 + pi/4) (footnote to Eq. bgkequation; the
 * printed bracket is misplaced, the diagonals are (1,1),(-1,1),(-1,-1),(1,-1)).
 * Weights 4/9, 1/9, 1/36 (Sec. 6.1, after Eq. standardequilibrium). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static double W9(int q) { return q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
/* D2Q5: v0 = 0 and v1..v4 as above; weights 1/3 and 1/6 (Sec. 6.1, D2Q5). */
static double W5(int q) { return q == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }

static int wrap(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Sec. 6.2, Eq. 1Dkernel: delta1D(r) = (1 + cos(pi |r| / 2)) / 4 for |r| <= 2. */
double orc_delta1d(double r) {
    double a = fabs(r);
    if (a > 2.0) return 0.0;
    return 0.25 * (1.0 + cos(M_PI * a / 2.0));
}

/* Lower-left node of the 4x4 support of a point at coordinate X: the nodes
 * floor(X)-1 .. floor(X)+2 are the only ones with |node - X| <= 2 that can
 * carry weight (at integer X the far node has r = 2 and weight 0). */
static int support_base(double X) { return (int)floor(X) - 1; }

/* ------------------------------------------------------------------------- */
/* Polygon forces on the vertices.
 * Hookean membrane springs (Sec. 3.2.3, BioSolverHookeanMembraneTension; the
 * same spring form as Eq. celljunctionforce): for the edge from vertex l to
 * its successor m, d = X_m - X_l, the force k_l (|d| - L0_l) d/|d| acts on l
 * and its opposite on m.
 * Internal pressure p (a term of the measured workloads, not of the paper):
 * F_l = p dA/dX_l = (p/2) (y_{l+1} - y_{l-1}, x_{l-1} - x_{l+1}) for a CCW
 * polygon of area A; it points outward.  F has shape (V, 2). */
void orc_polygon_forces(int nc, const int32_t* off, const double* xy, const double* L0,
                        const double* k, const double* p, double* F) {
    int V = off[nc];
    for (int l = 0; l < 2 * V; ++l) F[l] = 0.0;
    for (int c = 0; c < nc; ++c) {
        int a = off[c], b = off[c + 1], n = b - a;
        for (int t = 0; t < n; ++t) {
            int l = a + t, m = a + (t + 1) % n;
            double dx = xy[2 * m] - xy[2 * l];
            double dy = xy[2 * m + 1] - xy[2 * l + 1];
            double len = sqrt(dx * dx + dy * dy);
            double s = k[l] * (len - L0[l]) / len;
            F[2 * l] += s * dx;
            F[2 * l + 1] += s * dy;
            F[2 * m] -= s * dx;
            F[2 * m + 1] -= s * dy;
        }
        for (int t = 0; t < n; ++t) {
            int l = a + t, nx_ = a + (t + 1) % n, pv = a + (t + n - 1) % n;
            F[2 * l] += 0.5 * p[c] * (xy[2 * nx_ + 1] - xy[2 * pv + 1]);
            F[2 * l + 1] += 0.5 * p[c] * (xy[2 * pv] - xy[2 * nx_]);
        }
    }
}

/* Constant membrane tension, Eq. membraneforce (Sec. 3.2.3): for each vertex,
 * phi_m times the sum of the unit vectors towards its two neighbours.  Added
 * to F (does not clear it). */
void orc_tension_forces(int nc, const int32_t* off, const double* xy, double phim, double* F) {
    for (int c = 0; c < nc; ++c) {
        int a = off[c], n = off[c + 1] - a;
        for (int t = 0; t < n; ++t) {
            int l = a + t, pv = a + (t + n - 1) % n, nx_ = a + (t + 1) % n;
            double ax = xy[2 * pv] - xy[2 * l], ay = xy[2 * pv + 1] - xy[2 * l + 1];
            double bx = xy[2 * nx_] - xy[2 * l], by = xy[2 * nx_ + 1] - xy[2 * l + 1];
            double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by);
            F[2 * l] += phim * (ax / la + bx / lb);
            F[2 * l + 1] += phim * (ay / la + by / lb);
        }
    }
}

/* Cell junctions, Eq. celljunctionforce (Sec. 3.2.4).  Reading c28: when
 * the junctions are renewed, every membrane point i takes as partner the
 * closest membrane point j of another cell with |x_j - x_i| < l_max
 * (distance in FP64 with the periodic minimum image in x, and in y unless
 * there are walls; ties to the lower index), or none; between renewals the
 * partners are kept and the force is evaluated from the current positions:
 *   F_i += k_j (x_j - x_i)/|x_j - x_i| (|x_j - x_i| - l_0)  if |x_j - x_i| < l_max.
 * The force acts on i only, as the equation states. */
static void min_image(double* dx, double* dy, int nx, int ny, int bc_y) {
    *dx -= (double)nx * round(*dx / (double)nx);
    if (bc_y == 0) *dy -= (double)ny * round(*dy / (double)ny);
}

void orc_junction_partners(int nx, int ny, int bc_y, int nc, const int32_t* off,
                           const double* xy, double lmax, int32_t* partner) {
    int V = nc > 0 ? off[nc] : 0;
    int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * (V > 0 ? V : 1));
    for (int c = 0; c < nc; ++c)
        for (int l = off[c]; l < off[c + 1]; ++l) cell[l] = c;
    for (int i = 0; i < V; ++i) {
        int best = -1;
        double bd2 = lmax * lmax;
        for (int j = 0; j < V; ++j) {
            if (cell[j] == cell[i]) continue;
            double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
            min_image(&dx, &dy, nx, ny, bc_y);
            double d2 = dx * dx + dy * dy;
            if (d2 < bd2) {  /* j ascending: a tie keeps the lower index */
                bd2 = d2;
                best = j;
            }
        }
        partner[i] = best;
    }
    free(cell);
}

void orc_junction_forces(int nx, int ny, int bc_y, int nv, const double* xy,
                         const int32_t* partner, double k, double l0, double lmax, double* F) {
    for (int i = 0; i < nv; ++i) {
        int j = partner[i];
        if (j < 0) continue;
        double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
        min_image(&dx, &dy, nx, ny, bc_y);
        double L = sqrt(dx * dx + dy * dy);
        if (L < lmax && L > 0.0) {
            F[2 * i] += k * dx / L * (L - l0);
            F[2 * i + 1] += k * dy / L * (L - l0);
        }
    }
}

/* Per-cell polygon area by the shoelace formula, taken relative to the
 * cell's first vertex (the same quantity, better conditioned for large
 * coordinates) -- GeometryHandler::computeAreas, Sec. 3.3. */
void orc_cell_areas(int nc, const int32_t* off, const double* xy, double* area) {
    for (int c = 0; c < nc; ++c) {
        int a = off[c], n = off[c + 1] - a;
        double x0 = xy[2 * a], y0 = xy[2 * a + 1], s = 0.0;
        for (int t = 0; t < n; ++t) {
            int l = a + t, m = a + (t + 1) % n;
            double xl = xy[2 * l] - x0, yl = xy[2 * l + 1] - y0;
            double xm = xy[2 * m] - x0, ym = xy[2 * m + 1] - y0;
            s += xl * ym - xm * yl;
        }
        area[c] = 0.5 * s;
    }
}

/* ------------------------------------------------------------------------- */
/* Lattice labelling (Fig. 2: the domainID of the lattice nodes is set from
 * the polygons).  Reading: a node belongs to a cell when its centre is inside
 * the polygon by the crossing-number rule, half-open in y -- an edge a->b
 * crosses the row of the node when (y_a <= y) != (y_b <= y), and counts when
 * x < x_a + (y - y_a)(x_b - x_a)/(y_b - y_a).  The paper gives no rule for
 * overlapping polygons (its cells partition the tissue); reading taken: the
 * node's domainID is the lower cell index, and the node receives the sources
 * of every cell that contains it (the bitwise OR of their source flags).
 * Coordinates are unwrapped; the node index is taken modulo the periodic
 * sizes, rows outside a walled domain are skipped.
 * id[N]: 0 outside, c+1 for the lowest cell c containing the node.
 * src[N]: OR of the src_flag of the cells containing the node. */
void orc_rasterize(int nx, int ny, int bc_y, int nc, const int32_t* off, const double* xy,
                   const uint8_t* src_flag, int32_t* id, uint8_t* src) {
    long N = (long)nx * ny;
    for (long t = 0; t < N; ++t) { id[t] = 0; src[t] = 0; }
    for (int c = 0; c < nc; ++c) {
        int a = off[c], n = off[c + 1] - a;
        double xmin = xy[2 * a], xmax = xmin, ymin = xy[2 * a + 1], ymax = ymin;
        for (int t = 1; t < n; ++t) {
            double x = xy[2 * (a + t)], y = xy[2 * (a + t) + 1];
            if (x < xmin) xmin = x;
            if (x > xmax) xmax = x;
            if (y < ymin) ymin = y;
            if (y > ymax) ymax = y;
        }
        for (int J = (int)floor(ymin); J <= (int)ceil(ymax); ++J) {
            if (bc_y == 1 && (J < 0 || J >= ny)) continue;
            for (int I = (int)floor(xmin); I <= (int)ceil(xmax); ++I) {
                double xn = (double)I, yn = (double)J;
                int inside = 0;
                for (int t = 0; t < n; ++t) {
                    int l = a + t, m = a + (t + 1) % n;
                    double xa = xy[2 * l], ya = xy[2 * l + 1], xb = xy[2 * m], yb = xy[2 * m + 1];
                    if ((ya <= yn) != (yb <= yn)) {
                        double xc = xa + (yn - ya) * (xb - xa) / (yb - ya);
                        if (xn < xc) inside = !inside;
                    }
                }
                if (!inside) continue;
                long idx = (long)wrap(J, ny) * nx + wrap(I, nx);
                if (id[idx] == 0) id[idx] = c + 1;
                src[idx] |= src_flag[c];
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Force spreading, Eq. forcedistribution with the 4x4 kernel of Eq. 1Dkernel:
 * f(x) += F_l delta1D(x - X_l) delta1D(y - Y_l) (the two-dimensional kernel is
 * the product of the 1-D kernel in each axis; the printed delta1D(r)delta1D(r)
 * is read that way).  F_l is a per-vertex force, h = 1.  Serial, vertex
 * order.  Adds into fx, fy. */
void orc_spread(int nx, int ny, int bc_y, int nv, const double* xy, const double* F,
                double* fx, double* fy) {
    for (int l = 0; l < nv; ++l) {
        double X = xy[2 * l], Y = xy[2 * l + 1];
        int i0 = support_base(X), j0 = support_base(Y);
        for (int b = 0; b < 4; ++b) {
            int J = j0 + b;
            if (bc_y == 1 && (J < 0 || J >= ny)) continue;
            double wy = orc_delta1d((double)J - Y);
            for (int a = 0; a < 4; ++a) {
                int I = i0 + a;
                double w = orc_delta1d((double)I - X) * wy;
                long idx = (long)wrap(J, ny) * nx + wrap(I, nx);
                fx[idx] += F[2 * l] * w;
                fy[idx] += F[2 * l + 1] * w;
            }
        }
    }
}

/* Velocity interpolation, Eq. conversion2: U_l = sum_x u(x) delta(x - X_l). */
void orc_interp(int nx, int ny, int bc_y, int nv, const double* xy, const double* ux,
                const double* uy, double* U) {
    for (int l = 0; l < nv; ++l) {
        double X = xy[2 * l], Y = xy[2 * l + 1];
        int i0 = support_base(X), j0 = support_base(Y);
        double sx = 0.0, sy = 0.0;
        for (int b = 0; b < 4; ++b) {
            int J = j0 + b;
            if (bc_y == 1 && (J < 0 || J >= ny)) continue;
            double wy = orc_delta1d((double)J - Y);
            for (int a = 0; a < 4; ++a) {
                int I = i0 + a;
                double w = orc_delta1d((double)I - X) * wy;
                long idx = (long)wrap(J, ny) * nx + wrap(I, nx);
                sx += ux[idx] * w;
                sy += uy[idx] * w;
            }
        }
        U[2 * l] = sx;
        U[2 * l + 1] = sy;
    }
}

/* ------------------------------------------------------------------------- */
/* Streaming by pulling: the population q arriving at (i,j) left (i-cx, j-cy)
 * after the previous collision (left-hand side of Eq. bgkequation).  With
 * walls (reading c13: half-way bounce-back, the fluid walls are not described
 * in the paper), a population whose source row lies outside the domain is the
 * opposite population of the same node reflected back. */
static double pull(const double* post, const int* opp, int q, int i, int j, int nx, int ny,
                   int bc_y) {
    long N = (long)nx * ny;
    int si = wrap(i - CX[q], nx), sj = j - CY[q];
    if (sj < 0 || sj >= ny) {
        if (bc_y == 1) return post[(long)opp[q] * N + (long)j * nx + i];
        sj = wrap(sj, ny);
    }
    return post[(long)q * N + (long)sj * nx + si];
}

/* Species streaming with the membrane no-flux condition (Sec. 6.1,
 * "No-flux Boundary Condition for Reaction-Advection-Diffusion Equations").
 * A species confined to its domain (labels dom, one per node; equal labels =
 * one domain) does not take the population that would arrive at x along v_q
 * from a node x - v_q of another domain: that population is missing.
 *
 * Scheme 0, the paper's (reading c26): the missing population is the D2Q5
 * equilibrium w_q (phi + 3 v_q . j) of a density and a momentum (first
 * moment j = sum_k v_k g_k) obtained from the fluid of the domain:
 *   - the momentum is interpolated linearly between the fluid node
 *     y1 = x + v_q (in the direction the missing population travels) and
 *     zero at the wall point; the membrane sits at the half-way point
 *     x - v_q/2 of the crossing link (the static domain plane carries no
 *     finer position), so x lies at distance 1/2 from the wall and y1 at
 *     3/2: j(x) = (1/2)/(3/2) j(y1) = j(y1)/3;
 *   - the density is extrapolated linearly from the fluid nodes y1 and
 *     y2 = x + 2 v_q: phi(x) = 2 phi(y1) - phi(y2);
 *   - the densities and momenta of the fluid nodes are those of the
 *     previous step (mom: phi, jx, jy of the pulled populations before the
 *     collision, per node), so no population of the step depends on
 *     another one of the same step;
 *   - where y2 is not in the domain (or beyond a wall) the density is
 *     taken from y1 alone (zeroth order); where y1 is not in the domain
 *     either, the momentum is zero (walls on both sides of x) and the
 *     density is the node's own of the previous step.
 * The closure is first order in space, as the paper states for it, and it
 * does not conserve each domain's mass exactly.
 * Scheme 1 (not the paper's; kept as an option): half-way bounce-back, the
 * missing population is the opposite population of x itself, so nothing
 * crosses the membrane and each domain keeps its mass exactly.
 * Membranes that move (noflux_dynamic, reading c31) always use scheme 1.
 * Walls in y bounce back first (reading c13). */
static int in_domain(const int32_t* dom, int i, int j, int nx, int ny, int bc_y, int32_t d0) {
    if (j < 0 || j >= ny) {
        if (bc_y == 1) return 0;
        j = wrap(j, ny);
    }
    return dom[(long)j * nx + wrap(i, nx)] == d0;
}

static double pull_species(const orc_params* P, const double* post, const int* opp, int q,
                           int i, int j, const int32_t* dom, int confined, const double* mom,
                           int s) {
    int nx = P->nx, ny = P->ny, bc_y = P->bc_y;
    if (!confined || !dom || q == 0) return pull(post, opp, q, i, j, nx, ny, bc_y);
    long N = (long)nx * ny;
    int si = wrap(i - CX[q], nx), sj = j - CY[q];
    if (sj < 0 || sj >= ny) {
        if (bc_y == 1) return post[(long)opp[q] * N + (long)j * nx + i];
        sj = wrap(sj, ny);
    }
    int32_t d0 = dom[(long)j * nx + i];
    if (dom[(long)sj * nx + si] == d0) return post[(long)q * N + (long)sj * nx + si];
    if (P->noflux_dynamic || P->noflux_scheme == 1 || !mom)
        return post[(long)opp[q] * N + (long)j * nx + i];
    /* scheme 0: the equilibrium closure */
    const double* mphi = mom + (long)(3 * s) * N;
    const double* mjx = mphi + N;
    const double* mjy = mphi + 2 * N;
    int in1 = in_domain(dom, i + CX[q], j + CY[q], nx, ny, bc_y, d0);
    int in2 = in1 && in_domain(dom, i + 2 * CX[q], j + 2 * CY[q], nx, ny, bc_y, d0);
    long x0 = (long)j * nx + i;
    long x1 = (long)wrap(j + CY[q], ny) * nx + wrap(i + CX[q], nx);
    long x2 = (long)wrap(j + 2 * CY[q], ny) * nx + wrap(i + 2 * CX[q], nx);
    double phih, jh;
    if (in2) {
        phih = 2.0 * mphi[x1] - mphi[x2];
        jh = (CX[q] * mjx[x1] + CY[q] * mjy[x1]) / 3.0;
    } else if (in1) {
        phih = mphi[x1];
        jh = (CX[q] * mjx[x1] + CY[q] * mjy[x1]) / 3.0;
    } else {
        phih = mphi[x0];
        jh = 0.0;
    }
    return W5(q) * (phih + 3.0 * jh);
}

/* Density and momentum of every species from populations g (5S planes) at
 * the same node (no streaming): mom[3s], mom[3s+1], mom[3s+2] = phi, jx, jy.
 * The moments a run starts from: those of its initial populations. */
void orc_species_moments(const orc_params* P, const double* g, double* mom) {
    long N = (long)P->nx * P->ny;
    for (int s = 0; s < P->n_species; ++s) {
        const double* G = g + (long)5 * s * N;
        double* m = mom + (long)3 * s * N;
        for (long t = 0; t < N; ++t) {
            double phi = 0.0, jx = 0.0, jy = 0.0;
            for (int q = 0; q < 5; ++q) {
                phi += G[(long)q * N + t];
                jx += CX[q] * G[(long)q * N + t];
                jy += CY[q] * G[(long)q * N + t];
            }
            m[t] = phi;
            m[N + t] = jx;
            m[2 * N + t] = jy;
        }
    }
}

/* The reaction rate of species s at a node (reading c10: evaluated on the
 * pre-collision phi of the node, added after collision):
 *   react_model 0:  R_s = sum_b react[s][b] phi_b - decay[s] phi_s
 *   react_model 1:  the Schnakenberg system of the Turing-patterning example
 *                   (Sec. 4.2), receptor R = species 0, ligand L = species 1:
 *                   R_0 = gamma (a - R + R^2 L),  R_1 = gamma (b - R^2 L);
 *                   further species linear as above
 * plus src_rate[s] at nodes inside a source cell of species s. */
static double reaction(const orc_params* P, int s, const double* phi, int S, uint8_t srcbits) {
    double R;
    if (P->react_model == 1 && S >= 2 && s < 2) {
        double r2l = phi[0] * phi[0] * phi[1];
        R = s == 0 ? P->schnak[0] * (P->schnak[1] - phi[0] + r2l)
                   : P->schnak[0] * (P->schnak[2] - r2l);
    } else {
        R = -P->decay[s] * phi[s];
        for (int b = 0; b < S; ++b) R += P->react[s][b] * phi[b];
    }
    if ((srcbits >> s) & 1) R += P->src_rate[s];
    return R;
}

/* One lattice update: stream, then collide (Sec. 6.1).
 * Fluid, Eq. bgkequation with the equilibrium of Eq. standardequilibrium read
 * as the standard second-order polynomial
 *   f_eq = w rho [1 + 3 v.u + 9/2 (v.u)^2 - 3/2 u.u]   (c_s^2 = 1/3).
 * Moments rho = sum f, rho u = sum f v.  The body force f(x) from the spread:
 *   forcing 0 (Guo, Zheng & Shi 2002, the form the measured method uses):
 *     u = (sum f v + F/2) / rho,
 *     S_q = (1 - 1/(2 tau)) w_q [3 (v_q - u) + 9 (v_q.u) v_q] . F
 *   forcing 1 (the paper's term, He 1997, F a force density):
 *     u = sum f v / rho,  S_q = 3 w_q v_q . F
 *   f*_q = f_q - (f_q - f_eq_q)/tau + S_q.
 * Species s (D2Q5, Sec. 6.1): g_eq = phi w (1 + 3 v.u) with the fluid u,
 *   phi = sum g, tau_D = 3 D + 1/2 (D = c_s^2 (tau_D - 1/2), c_s^2 = 1/3 for
 *   weights 1/3, 1/6), g*_q = g_q - (g_q - g_eq_q)/tau_D + w_q R_s with the
 *   reaction (reading c10: added after collision, evaluated on the
 *   pre-collision phi of the same node)
 *   R_s = sum_b react[s][b] phi_b - decay[s] phi_s + src_rate[s] [src bit s].
 * Walls bounce species back too (zero flux); the membranes between
 * domains of a confined species take the no-flux closure (pull_species).
 * Internal pressure nodes (Sec. 6.1, pressure boundary condition; reading
 * c30): where pmask is set, every pulled population is multiplied by
 * gamma = pressure_rho / rho before the moments are taken, so the node holds
 * the prescribed density and keeps its velocity (gamma cancels in u).
 * Mass sources (Sec. 3.2.3; reading c29): msrc[x] is added to the node's
 * mass after the collision, spread over the directions by the weights,
 * f*_q += w_q msrc[x], which adds no momentum.  With lab (cell labels, > 0
 * inside a cell) the source of a node inside a cell gains mass_beta phi_s
 * (s = mass_species; reading c32: the concentration-proportional source of
 * the validation Case III, on the pre-collision phi of the node).
 * fpost_*: 9 planes of N; gpost_*: S*5 planes; fx, fy may be NULL (no force);
 * rho, ux, uy, phi (S planes) may be NULL; msrc, pmask, lab may be NULL.
 * mom_in (3S planes: phi, jx, jy per species): the moments of the previous
 * step for the no-flux closure of the confined species; mom_out receives
 * this step's (either may be NULL). */
void orc_lattice_step(const orc_params* P, const double* fpost_in, double* fpost_out,
                      const double* gpost_in, double* gpost_out, const double* fx,
                      const double* fy, const uint8_t* src, double* rho_out, double* ux_out,
                      double* uy_out, double* phi_out, const int32_t* dom, const double* msrc,
                      const uint8_t* pmask, const int32_t* lab, const double* mom_in,
                      double* mom_out) {
    int nx = P->nx, ny = P->ny, S = P->n_species;
    long N = (long)nx * ny;
    double tau = P->tau;
    static const int OPP5[5] = {0, 3, 4, 1, 2};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long idx = (long)j * nx + i;
            double f[9];
            for (int q = 0; q < 9; ++q) f[q] = pull(fpost_in, OPP, q, i, j, nx, ny, P->bc_y);
            /* the species' pulled populations and concentrations (needed by
             * the concentration-proportional mass source) */
            double g[4][5], phi[4];
            for (int s = 0; s < S; ++s) {
                phi[s] = 0.0;
                for (int q = 0; q < 5; ++q) {
                    g[s][q] = pull_species(P, gpost_in + (long)s * 5 * N, OPP5, q, i, j, dom,
                                           (P->noflux >> s) & 1, mom_in, s);
                    phi[s] += g[s][q];
                }
                if (mom_out) {  /* this step's moments, for the next step's closures */
                    mom_out[(long)(3 * s) * N + idx] = phi[s];
                    mom_out[(long)(3 * s + 1) * N + idx] = g[s][1] - g[s][3];
                    mom_out[(long)(3 * s + 2) * N + idx] = g[s][2] - g[s][4];
                }
            }
            const int beta_on = lab && lab[idx] > 0 && P->mass_beta != 0.0 &&
                                P->mass_species >= 0 && P->mass_species < S;
            double Sm = msrc ? msrc[idx] : 0.0;
            if (beta_on) Sm += P->mass_beta * phi[P->mass_species];
            double rho = 0.0, jx = 0.0, jy = 0.0;
            if (pmask && pmask[idx]) {
                for (int q = 0; q < 9; ++q) rho += f[q];
                double gam = P->pressure_rho / rho;
                for (int q = 0; q < 9; ++q) f[q] *= gam;
                rho = 0.0;
            }
            for (int q = 0; q < 9; ++q) {
                rho += f[q];
                jx += f[q] * CX[q];
                jy += f[q] * CY[q];
            }
            double Fx = fx ? fx[idx] : 0.0, Fy = fy ? fy[idx] : 0.0;
            double ux, uy;
            if (P->forcing == 0) {
                ux = (jx + 0.5 * Fx) / rho;
                uy = (jy + 0.5 * Fy) / rho;
            } else {
                ux = jx / rho;
                uy = jy / rho;
            }
            double usq = ux * ux + uy * uy;
            for (int q = 0; q < 9; ++q) {
                double vu = CX[q] * ux + CY[q] * uy;
                double feq = W9(q) * rho * (1.0 + 3.0 * vu + 4.5 * vu * vu - 1.5 * usq);
                double Sq;
                if (P->forcing == 0)
                    Sq = (1.0 - 0.5 / tau) * W9(q) *
                         (3.0 * ((CX[q] - ux) * Fx + (CY[q] - uy) * Fy) +
                          9.0 * vu * (CX[q] * Fx + CY[q] * Fy));
                else
                    Sq = 3.0 * W9(q) * (CX[q] * Fx + CY[q] * Fy);
                if (msrc || beta_on) Sq += W9(q) * Sm;
                fpost_out[(long)q * N + idx] = f[q] - (f[q] - feq) / tau + Sq;
            }
            if (rho_out) rho_out[idx] = rho;
            if (ux_out) ux_out[idx] = ux;
            if (uy_out) uy_out[idx] = uy;

            for (int s = 0; s < S; ++s) {
                double R = reaction(P, s, phi, S, src ? src[idx] : 0);
                double tauD = 3.0 * P->D[s] + 0.5;
                for (int q = 0; q < 5; ++q) {
                    double vu = CX[q] * ux + CY[q] * uy;
                    double geq = phi[s] * W5(q) * (1.0 + 3.0 * vu);
                    gpost_out[((long)s * 5 + q) * N + idx] =
                        g[s][q] - (g[s][q] - geq) / tauD + W5(q) * R;
                }
                if (phi_out) phi_out[(long)s * N + idx] = phi[s];
            }
        }
    }
}

/* Species-only update with a frozen velocity field (u = 0 when ux, uy are
 * NULL): the D2Q5 part of orc_lattice_step, used by the steady solve. */
void orc_species_step(const orc_params* P, const double* gpost_in, double* gpost_out,
                      const double* ux_in, const double* uy_in, const uint8_t* src,
                      double* phi_out, const int32_t* dom, const double* mom_in,
                      double* mom_out) {
    int nx = P->nx, ny = P->ny, S = P->n_species;
    long N = (long)nx * ny;
    static const int OPP5[5] = {0, 3, 4, 1, 2};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            long idx = (long)j * nx + i;
            double ux = ux_in ? ux_in[idx] : 0.0, uy = uy_in ? uy_in[idx] : 0.0;
            double g[4][5], phi[4];
            for (int s = 0; s < S; ++s) {
                phi[s] = 0.0;
                for (int q = 0; q < 5; ++q) {
                    g[s][q] = pull_species(P, gpost_in + (long)s * 5 * N, OPP5, q, i, j, dom,
                                           (P->noflux >> s) & 1, mom_in, s);
                    phi[s] += g[s][q];
                }
                if (mom_out) {
                    mom_out[(long)(3 * s) * N + idx] = phi[s];
                    mom_out[(long)(3 * s + 1) * N + idx] = g[s][1] - g[s][3];
                    mom_out[(long)(3 * s + 2) * N + idx] = g[s][2] - g[s][4];
                }
            }
            for (int s = 0; s < S; ++s) {
                double R = reaction(P, s, phi, S, src ? src[idx] : 0);
                double tauD = 3.0 * P->D[s] + 0.5;
                for (int q = 0; q < 5; ++q) {
                    double vu = CX[q] * ux + CY[q] * uy;
                    double geq = phi[s] * W5(q) * (1.0 + 3.0 * vu);
                    gpost_out[((long)s * 5 + q) * N + idx] =
                        g[s][q] - (g[s][q] - geq) / tauD + W5(q) * R;
                }
                if (phi_out) phi_out[(long)s * N + idx] = phi[s];
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* The coupled time step, in the order of Fig. 1: from the geometry X^n the
 * vertex forces F^n are computed and spread to the lattice; the fluid (and
 * the species, which receive the fluid velocity and the cell labels) is
 * advanced one step; the velocity u^n is interpolated back to the vertices
 * and they move by forward Euler, X^{n+1} = X^n + U^n (first order explicit,
 * Sec. 3.4).  Labels are recomputed from X^n at the start of each step.
 *
 * State in/out: xy (V,2), f (9 planes, post-collision), g (5S planes).
 * Outputs of the last step (any may be NULL): rho, ux, uy, phi (S planes),
 * id, src, fx, fy (the spread force), Fv (V,2 vertex forces).
 * tension: constant membrane tension magnitude (0 = off).  dom: static domain
 * labels for the confined species (NULL = none; see pull_species).
 * Mass sources (Sec. 3.2.3, reading c29): with mrate (per cell, NULL = none)
 * every node labelled with cell c receives
 *   S_c = mrate[c] + mass_alpha (marea[c] - A_c(X^n))
 * (the proportional area controller; without marea S_c = mrate[c]), A_c the
 * polygon area of Sec. 3.3 at the start of the step; with mass_beta != 0 a
 * node inside a cell also gains mass_beta phi_s (reading c32).  With
 * noflux_dynamic the confined species are bounded by the cells' labels of
 * each step (id: 0 outside, c+1 inside) instead of dom (reading c31: the
 * membranes move).  nsrc: a static mass
 * source per node (the field S(x,t) of Fig. 1; NULL = none), added to the
 * cells' sources (a point source is one node of it).  pmask: internal
 * pressure nodes (NULL = none; see orc_lattice_step).  mom (3S planes,
 * in/out, may be NULL): the species moments of the previous step that the
 * no-flux closure reads (pull_species); NULL starts from the moments of the
 * initial populations. */
int orc_run(const orc_params* P, int nc, const int32_t* off, double* xy, const double* L0,
            const double* k, const double* p, double tension, const uint8_t* src_flag,
            int n_steps, double* f, double* g, double* rho, double* ux, double* uy, double* phi,
            int32_t* id, uint8_t* src, double* fx, double* fy, double* Fv, const int32_t* dom,
            const double* mrate, const double* marea, const uint8_t* pmask, const double* nsrc,
            double* mom) {
    int nx = P->nx, ny = P->ny, S = P->n_species;
    long N = (long)nx * ny;
    int V = nc > 0 ? off[nc] : 0;
    double* f2 = (double*)malloc(sizeof(double) * 9 * N);
    double* g2 = (double*)malloc(sizeof(double) * (S > 0 ? 5 * S * N : 1));
    double* Fx = (double*)malloc(sizeof(double) * N);
    double* Fy = (double*)malloc(sizeof(double) * N);
    double* Ux = (double*)malloc(sizeof(double) * N);
    double* Uy = (double*)malloc(sizeof(double) * N);
    double* F = (double*)malloc(sizeof(double) * 2 * (V > 0 ? V : 1));
    double* U = (double*)malloc(sizeof(double) * 2 * (V > 0 ? V : 1));
    int32_t* lid = (int32_t*)malloc(sizeof(int32_t) * N);
    uint8_t* lsrc = (uint8_t*)malloc(N);
    int32_t* partner = (int32_t*)malloc(sizeof(int32_t) * (V > 0 ? V : 1));
    double* Sn = (mrate || nsrc) ? (double*)malloc(sizeof(double) * N) : NULL;
    double* Sc = (double*)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    if (!f2 || !g2 || !Fx || !Fy || !Ux || !Uy || !F || !U || !lid || !lsrc || !partner || !Sc ||
        ((mrate || nsrc) && !Sn))
        return -1;
    for (int l = 0; l < V; ++l) partner[l] = -1;
    /* the species moments of the previous step, for the no-flux closure:
     * carried in mom (3S planes) across calls, else those of the initial
     * populations */
    double *ma = NULL, *mb = NULL;
    if (S > 0 && P->noflux) {
        ma = (double*)malloc(sizeof(double) * 3 * S * N);
        mb = (double*)malloc(sizeof(double) * 3 * S * N);
        if (!ma || !mb) return -1;
        if (mom) memcpy(ma, mom, sizeof(double) * 3 * S * N);
        else orc_species_moments(P, g, ma);
    }
    double *fa = f, *fb = f2, *ga = g, *gb = g2;
    for (int n = 0; n < n_steps; ++n) {
        int last = (n == n_steps - 1);
        orc_rasterize(nx, ny, P->bc_y, nc, off, xy, src_flag, lid, lsrc);
        if (V > 0) {
            orc_polygon_forces(nc, off, xy, L0, k, p, F);
            if (tension != 0.0) orc_tension_forces(nc, off, xy, tension, F);
            if (P->junction_period > 0) {
                if (n % P->junction_period == 0)
                    orc_junction_partners(nx, ny, P->bc_y, nc, off, xy, P->junction_lmax, partner);
                orc_junction_forces(nx, ny, P->bc_y, V, xy, partner, P->junction_k,
                                    P->junction_l0, P->junction_lmax, F);
            }
        }
        for (long t = 0; t < N; ++t) { Fx[t] = 0.0; Fy[t] = 0.0; }
        if (V > 0) orc_spread(nx, ny, P->bc_y, V, xy, F, Fx, Fy);
        if (mrate) {
            if (marea) orc_cell_areas(nc, off, xy, Sc);
            for (int c = 0; c < nc; ++c)
                Sc[c] = marea ? mrate[c] + P->mass_alpha * (marea[c] - Sc[c]) : mrate[c];
            for (long t = 0; t < N; ++t) Sn[t] = lid[t] > 0 ? Sc[lid[t] - 1] : 0.0;
        } else if (nsrc) {
            for (long t = 0; t < N; ++t) Sn[t] = 0.0;
        }
        if (nsrc)
            for (long t = 0; t < N; ++t) Sn[t] += nsrc[t];
        orc_lattice_step(P, fa, fb, ga, gb, Fx, Fy, lsrc, last ? rho : NULL, Ux, Uy,
                         last ? phi : NULL, P->noflux_dynamic ? lid : dom, Sn, pmask,
                         P->mass_beta != 0.0 ? lid : NULL, ma, mb);
        if (V > 0) {
            orc_interp(nx, ny, P->bc_y, V, xy, Ux, Uy, U);
            if (last && Fv) memcpy(Fv, F, sizeof(double) * 2 * V);
            for (int l = 0; l < 2 * V; ++l) xy[l] += U[l];
        }
        if (last) {
            if (ux) memcpy(ux, Ux, sizeof(double) * N);
            if (uy) memcpy(uy, Uy, sizeof(double) * N);
            if (id) memcpy(id, lid, sizeof(int32_t) * N);
            if (src) memcpy(src, lsrc, N);
            if (fx) memcpy(fx, Fx, sizeof(double) * N);
            if (fy) memcpy(fy, Fy, sizeof(double) * N);
        }
        double* t;
        t = fa; fa = fb; fb = t;
        t = ga; ga = gb; gb = t;
        t = ma; ma = mb; mb = t;
    }
    if (mom && ma) memcpy(mom, ma, sizeof(double) * 3 * S * N);
    free(ma); free(mb);
    if (fa != f) memcpy(f, fa, sizeof(double) * 9 * N);
    if (S > 0 && ga != g) memcpy(g, ga, sizeof(double) * 5 * S * N);
    free(f2); free(g2); free(Fx); free(Fy); free(Ux); free(Uy); free(F); free(U);
    free(lid); free(lsrc); free(partner); free(Sn); free(Sc);
    return 0;
}

/* Steady morphogen solve on a static labelling with u = 0: repeat the D2Q5
 * update until the residual r = max|phi^{n+1} - phi^n| / max|phi^{n+1}|
 * (reading c20 of the undefined "resid"), checked every `check_every` steps
 * on the last step pair, is <= tol, or max_steps is reached.
 * g (5S planes) in/out; phi (S planes) out; returns the steps taken. */
long orc_steady(const orc_params* P, const uint8_t* src, double* g, double tol, long max_steps,
                int check_every, double* phi, double* resid_out) {
    int S = P->n_species;
    long N = (long)P->nx * P->ny;
    double* g2 = (double*)malloc(sizeof(double) * 5 * S * N);
    double* p0 = (double*)malloc(sizeof(double) * S * N);
    double* p1 = (double*)malloc(sizeof(double) * S * N);
    double *ga = g, *gb = g2;
    double r = INFINITY;
    long n = 0;
    while (n < max_steps) {
        int check = ((n + 1) % check_every) == 0;
        orc_species_step(P, ga, gb, NULL, NULL, src, p0, NULL, NULL, NULL);
        double* t = ga; ga = gb; gb = t;
        ++n;
        if (check) {
            /* phi^{n+1}: the zeroth moment of the populations just streamed */
            orc_species_step(P, ga, gb, NULL, NULL, src, p1, NULL, NULL, NULL);
            double dmax = 0.0, pmax = 0.0;
            for (long x = 0; x < S * N; ++x) {
                double d = fabs(p1[x] - p0[x]);
                if (d > dmax) dmax = d;
                if (fabs(p1[x]) > pmax) pmax = fabs(p1[x]);
            }
            r = pmax > 0.0 ? dmax / pmax : (dmax > 0.0 ? INFINITY : 0.0);
            if (r <= tol) break;
        }
    }
    /* phi of the final state */
    orc_species_step(P, ga, gb, NULL, NULL, src, phi, NULL, NULL, NULL);
    if (ga != g) memcpy(g, ga, sizeof(double) * 5 * S * N);
    free(g2); free(p0); free(p1);
    if (resid_out) *resid_out = r;
    return n;
}

/* ------------------------------------------------------------------------- */
/* Convolution layers of the neural operator that warm-starts the steady
 * morphogen solve (a learned part the measured method adds; the paper has no
 * network).  Plain definitions in FP64, NHWC layout, 3x3 taps, zero padding:
 *   out[n,y,x,o] = b[o] + sum_{ky,kx,i} in[n,y+ky-1,x+kx-1,i] w[ky,kx,i,o]
 * dgrad: din[n,y,x,i] = sum_{ky,kx,o} dout[n,y-ky+1,x-kx+1,o] w[ky,kx,i,o]
 * wgrad: dw[ky,kx,i,o] = sum_{n,y,x} in[n,y+ky-1,x+kx-1,i] dout[n,y,x,o],
 *        db[o] = sum_{n,y,x} dout[n,y,x,o]. */
void orc_conv3x3(int N, int H, int W, int Ci, int Co, const double* in, const double* w,
                 const double* b, double* out) {
    for (int n = 0; n < N; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int o = 0; o < Co; ++o) {
                    double s = b ? b[o] : 0.0;
                    for (int ky = 0; ky < 3; ++ky) {
                        int yy = y + ky - 1;
                        if (yy < 0 || yy >= H) continue;
                        for (int kx = 0; kx < 3; ++kx) {
                            int xx = x + kx - 1;
                            if (xx < 0 || xx >= W) continue;
                            const double* ip = in + (((long)n * H + yy) * W + xx) * Ci;
                            const double* wp = w + ((long)(ky * 3 + kx) * Ci) * Co + o;
                            for (int i = 0; i < Ci; ++i) s += ip[i] * wp[(long)i * Co];
                        }
                    }
                    out[(((long)n * H + y) * W + x) * Co + o] = s;
                }
}

void orc_conv3x3_dgrad(int N, int H, int W, int Ci, int Co, const double* dout, const double* w,
                       double* din) {
    for (int n = 0; n < N; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int i = 0; i < Ci; ++i) {
                    double s = 0.0;
                    for (int ky = 0; ky < 3; ++ky) {
                        int yy = y - ky + 1;
                        if (yy < 0 || yy >= H) continue;
                        for (int kx = 0; kx < 3; ++kx) {
                            int xx = x - kx + 1;
                            if (xx < 0 || xx >= W) continue;
                            const double* gp = dout + (((long)n * H + yy) * W + xx) * Co;
                            const double* wp = w + (((long)(ky * 3 + kx) * Ci) + i) * Co;
                            for (int o = 0; o < Co; ++o) s += gp[o] * wp[o];
                        }
                    }
                    din[(((long)n * H + y) * W + x) * Ci + i] = s;
                }
}

void orc_conv3x3_wgrad(int N, int H, int W, int Ci, int Co, const double* in, const double* dout,
                       double* dw, double* db) {
    for (long t = 0; t < 9L * Ci * Co; ++t) dw[t] = 0.0;
    if (db)
        for (int o = 0; o < Co; ++o) db[o] = 0.0;
    for (int n = 0; n < N; ++n)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const double* gp = dout + (((long)n * H + y) * W + x) * Co;
                if (db)
                    for (int o = 0; o < Co; ++o) db[o] += gp[o];
                for (int ky = 0; ky < 3; ++ky) {
                    int yy = y + ky - 1;
                    if (yy < 0 || yy >= H) continue;
                    for (int kx = 0; kx < 3; ++kx) {
                        int xx = x + kx - 1;
                        if (xx < 0 || xx >= W) continue;
                        const double* ip = in + (((long)n * H + yy) * W + xx) * Ci;
                        double* wp = dw + ((long)(ky * 3 + kx) * Ci) * Co;
                        for (int i = 0; i < Ci; ++i)
                            for (int o = 0; o < Co; ++o) wp[(long)i * Co + o] += ip[i] * gp[o];
                    }
                }
            }
}
