/*
 * lbib.h -- C ABI of the GB300 (sm_103a) coupled lattice-Boltzmann /
 * immersed-boundary step of LBIBCell (Tanaka, Sichau & Iber,
 * arXiv:1503.06726).
 *
 * One context simulates one tissue on one GPU: a D2Q9 BGK fluid with a body
 * force (Sec. 6.1, Eq. bgkequation, Eq. standardequilibrium), up to four
 * D2Q5 advection-diffusion-reaction species that receive the fluid velocity
 * (Sec. 6.1, D2Q5 scheme), and closed polygon cells whose vertex forces are
 * spread to the lattice and whose vertices move with the interpolated fluid
 * velocity (Sec. 6.2, Eq. forcedistribution, Eq. conversion2, Eq. 1Dkernel;
 * the cycle of Fig. 1).
 *
 * Memory and threading rules common to every call:
 *   - All device memory is owned by the caller.  lbib_workspace_size() says
 *     how many bytes one context needs; the caller allocates them (any
 *     allocator; 256-byte alignment) and passes the pointer to
 *     lbib_create().  The library allocates no device memory of its own; it
 *     only mallocs the small host-side context header.
 *   - Host pointers passed in are read before the call returns; the caller
 *     keeps ownership.  Host output buffers are caller-allocated.
 *   - Work is enqueued on the CUDA stream given to lbib_create().
 *     lbib_step() and lbib_set_cell_params() are asynchronous; the other
 *     lbib_set_*() and lbib_get_*() calls synchronise that stream before
 *     they return.
 *   - A context must not be used from two host threads at once.
 *   - Every call returns LBIB_OK (0) or a negative LBIB_E_* code; no call
 *     aborts or throws.  lbib_last_error() gives a one-line reason.
 *
 * Lattice conventions: node (i, j) sits at position (i, j), i along x.
 * Fields returned to the host are dense nx*ny arrays, row-major in j (index
 * j*nx + i), in double precision whatever the storage precision.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBIB_OK 0
#define LBIB_E_PARAM (-1)       /* invalid parameter (size, tau <= 1/2, D <= 0, ...) */
#define LBIB_E_WORKSPACE (-2)   /* workspace pointer NULL, misaligned or too small */
#define LBIB_E_CELLS (-3)       /* invalid cell data (CSR, < 3 vertices, too many) */
#define LBIB_E_NONFINITE (-4)   /* a non-finite density or velocity appeared */
#define LBIB_E_TIMEOUT (-5)     /* a bounded device-side wait ran out */
#define LBIB_E_CUDA (-6)        /* a CUDA runtime call failed */
#define LBIB_E_STATE (-7)       /* call not valid in the context's current state */
#define LBIB_E_CHECK (-8)       /* checking build only: a kernel access failed its bounds
                                   or alignment check (it was skipped, not made) */

/* storage precision of the lattice populations */
#define LBIB_FP64 0   /* FP64 storage, FP64 arithmetic */
#define LBIB_FP32 1   /* FP32 storage of f - w rho0 (shifted), FP32 arithmetic */
#define LBIB_FP16 2   /* FP16 storage of (f - w rho0)/(w sigma), FP32 arithmetic */

/* reaction model of the species */
#define LBIB_REACT_LINEAR 0        /* R_s = sum_b react[s][b] phi_b - decay[s] phi_s */
#define LBIB_REACT_SCHNAKENBERG 1  /* species 0, 1 = receptor R, ligand L (Sec. 4.2):
                                      R_0 = gamma (a - R + R^2 L), R_1 = gamma (b - R^2 L) */

/* membrane no-flux scheme of the confined species (noflux_mask) */
#define LBIB_NOFLUX_CLOSURE 0     /* Sec. 6.1: the missing populations are equilibria of a
                                     density extrapolated from, and a momentum interpolated
                                     between, the fluid and the wall */
#define LBIB_NOFLUX_BOUNCEBACK 1  /* half-way bounce-back (exact mass per domain; not the
                                     paper's condition) */

/* body-force scheme */
#define LBIB_GUO 0        /* Guo, Zheng & Shi 2002: u = (sum f v + F/2)/rho */
#define LBIB_HE_PAPER 1   /* the paper's term of Eq. bgkequation, 3 w_i v_i.F */

/* lbib_get_fields() selection bits */
#define LBIB_RHO 1u
#define LBIB_U 2u
#define LBIB_PHI 4u
#define LBIB_X 8u
#define LBIB_AREA 16u
#define LBIB_ID 32u
#define LBIB_FORCE 64u
#define LBIB_VFORCE 128u

/* The global configuration of Sec. 3.1 (simulation size, viscosity through
 * tau, diffusion coefficients) plus the reaction terms of the species.
 *   nx, ny       lattice size (x periodic; y periodic or walls), >= 8 each;
 *                a plane (nx rounded up to a multiple of 64, times ny) must
 *                hold fewer than 2^31 nodes (kernels index planes in 32 bits)
 *   bc_y         0: periodic in y; 1: half-way bounce-back walls at y = -1/2
 *                and y = ny - 1/2 for the fluid and the species
 *   n_species    0..4 D2Q5 species
 *   tau          fluid relaxation time (> 1/2); nu = (tau - 1/2)/3
 *   rho0         reference density (initial state f = w rho0)
 *   D[s]         diffusion coefficient of species s (> 0); tau_D = 3 D + 1/2
 *   decay, react, src_rate: reaction rate of species s
 *                R_s = sum_b react[s][b] phi_b - decay[s] phi_s
 *                      + src_rate[s] * [the node lies in a cell whose
 *                                       src_flag has bit s set]
 *                (a node inside several overlapping cells takes the sources
 *                of all of them; the paper's cells do not overlap)
 *   forcing      LBIB_GUO or LBIB_HE_PAPER
 *   precision    LBIB_FP64, LBIB_FP32 or LBIB_FP16
 *   fp16_scale   sigma of the FP16 fluid storage (default 2^-10 when 0)
 *   fp16_scale_species  sigma of the FP16 species storage g/(w sigma)
 *                (default 2^-8 when 0)
 *   tension      constant membrane tension phi_m of Eq. membraneforce added
 *                to every vertex (0 = off)
 *   body_force   uniform body force density (fx, fy) added at every node on
 *                top of the spread cell forces (e.g. a channel driving force)
 *   reaction     LBIB_REACT_LINEAR, or LBIB_REACT_SCHNAKENBERG (needs two
 *                or more species; species 0 and 1 take the Schnakenberg
 *                rates of the Turing-patterning example, Sec. 4.2, with
 *                schnak = {gamma, a, b}; further species stay linear; the
 *                src_rate sources add to every species)
 *   noflux_mask  bit s: species s is confined to its domain: it does not
 *                cross the boundaries between the domains set with
 *                lbib_set_domains(); 0 = no domain plane
 *   noflux_scheme how a confined species meets a membrane.
 *                LBIB_NOFLUX_CLOSURE, the paper's no-flux condition (Sec. 6.1):
 *                a population that would arrive at x along v_q from another
 *                domain is replaced by the D2Q5 equilibrium
 *                w_q (phi^ + 3 v_q . j^) with phi^ = 2 phi(x + v_q) -
 *                phi(x + 2 v_q) (first-order extrapolation) and j^ the first
 *                moment at x + v_q scaled by 1/3 (first-order interpolation to
 *                zero at the half-way point of the link), moments of the
 *                previous step; first order, and each domain's mass is not
 *                kept exactly.  LBIB_NOFLUX_BOUNCEBACK: half-way bounce-back on
 *                every link between domains (each domain keeps its mass)
 *   junction_k, junction_l0, junction_lmax, junction_period
 *                cell junctions (Eq. celljunctionforce, Sec. 3.2.4): every
 *                junction_period steps (counted from lbib_set_cells or
 *                lbib_set_state; 0 = no junctions) each vertex takes as
 *                partner the closest vertex of another cell closer than
 *                junction_lmax (periodic minimum image, ties to the lower
 *                index); every step it receives the force
 *                junction_k (d/|d|)(|d| - junction_l0), d = X_partner - X,
 *                while |d| < junction_lmax.  Steps with junctions move the
 *                vertices and compute the forces in separate launches and
 *                are not captured in graphs.
 *   mass_sources, mass_alpha
 *                1 = per-cell mass sources (Sec. 3.2.3): every step each
 *                node labelled with cell c (the lowest cell containing it)
 *                gains S_c = rate_c + mass_alpha (A0_c - A_c) of fluid mass,
 *                added after the collision as w_q S_c in every direction (no
 *                momentum); A_c is the polygon area at the start of the
 *                step, rate_c and the set points A0_c come from
 *                lbib_set_mass_sources (the controller term only once set
 *                points are given).  The cells are labelled every step.
 *   pressure_nodes, pressure_rho
 *                1 = internal pressure nodes (Sec. 6.1): before the
 *                collision every population of a node flagged by
 *                lbib_set_pressure_nodes is multiplied by
 *                pressure_rho / rho, so the node holds the prescribed
 *                density (pressure rho/3) and keeps its velocity; such
 *                nodes take up or give off mass (the sink of growing
 *                tissues).  pressure_rho > 0.
 *   node_sources 1 = a static mass source per node (the field S(x,t) of
 *                Fig. 1; a point source is one node of it), set by
 *                lbib_set_node_sources and added to the cells' sources in
 *                the same way (w_q S after the collision). */
typedef struct lbib_params {
    int32_t nx, ny, bc_y, n_species;
    double tau, rho0;
    double D[4], decay[4], react[4][4], src_rate[4];
    int32_t forcing, precision;
    double fp16_scale, fp16_scale_species;
    double tension;
    double body_force[2];
    int32_t reaction, noflux_mask;
    double schnak[3];
    double junction_k, junction_l0, junction_lmax;
    int32_t junction_period, junction_pad;
    int32_t mass_sources, pressure_nodes;
    double mass_alpha, pressure_rho;
    int32_t node_sources, noflux_scheme;
} lbib_params;

typedef struct lbib_ctx lbib_ctx;

/* Bytes of device workspace one context needs for this lattice and at most
 * max_vertices vertices in max_cells cells.  Returns LBIB_E_PARAM for invalid
 * parameters. */
int lbib_workspace_size(const lbib_params* params, int32_t max_vertices, int32_t max_cells,
                        uint64_t* bytes_out);

/* Create a context over a caller-owned device workspace of `bytes` bytes
 * (256-byte aligned) and a CUDA stream (cudaStream_t passed as void*; NULL =
 * the legacy default stream).  Populations start at rest, f = w rho0, g = 0.
 * On success *out owns a small host header released by lbib_destroy(). */
int lbib_create(const lbib_params* params, int32_t max_vertices, int32_t max_cells,
                void* d_workspace, uint64_t bytes, void* cuda_stream, lbib_ctx** out);

/* Load the geometry and force description of the cells (the geometry and
 * force files of Sec. 3.1), all host arrays:
 *   cell_off   n_cells+1 int32, CSR offsets of each cell's vertices
 *   xy         2*V doubles, vertex positions (x, y), counter-clockwise per
 *              cell (Fig. 2), unwrapped (may leave [0, nx) in periodic axes)
 *   rest_len   V doubles, rest length of edge l -> next(l); NULL = the
 *              current edge lengths
 *   k_spring   V doubles, Hookean constant of edge l; NULL = 0
 *   pressure   n_cells doubles, internal pressure p (force p dA/dX); NULL = 0
 *   src_flag   n_cells bytes, bit s = the cell is a source of species s
 * Cells need 3 .. 1024 vertices.  Replaces any previous cells. */
int lbib_set_cells(lbib_ctx* ctx, int32_t n_cells, const int32_t* cell_off, const double* xy,
                   const double* rest_len, const double* k_spring, const double* pressure,
                   const uint8_t* src_flag);

/* Set the static domains of the confined species (noflux_mask): labels is a
 * host array of nx*ny int32, row-major in j, one label per node (any values;
 * neighbouring nodes with different labels are separated by a membrane; the
 * paper's static cellular domain is the cell index inside cells and one
 * common label outside).  NULL: one domain everywhere (nothing confined).
 * The domain plane lives in the workspace and is read by every lattice
 * update; it is zero (one domain) until set.  LBIB_E_STATE when the context
 * was created with noflux_mask 0.  Synchronises the context stream. */
int lbib_set_domains(lbib_ctx* ctx, const int32_t* labels);

/* Set the per-cell mass sources (mass_sources): rate (host, n_cells doubles,
 * NULL = 0) is the constant part of each cell's source, target_area (host,
 * n_cells doubles, NULL = controller off) the set points A0_c of the
 * proportional area controller S_c = rate_c + mass_alpha (A0_c - A_c)
 * (Sec. 3.2.3).  Both are copied; they apply from the next step on and stay
 * until set again.  LBIB_E_STATE when the context was created with
 * mass_sources 0.  Synchronises the context stream. */
int lbib_set_mass_sources(lbib_ctx* ctx, const double* rate, const double* target_area);

/* Set the internal pressure nodes (pressure_nodes): mask is a host array of
 * nx*ny bytes, row-major in j, nonzero = the node is held at pressure_rho
 * (Sec. 6.1).  NULL clears every node.  The plane lives in the workspace and
 * is zero until set.  LBIB_E_STATE when the context was created with
 * pressure_nodes 0.  Synchronises the context stream. */
int lbib_set_pressure_nodes(lbib_ctx* ctx, const uint8_t* mask);

/* Set the static mass source per node (node_sources): S is a host array of
 * nx*ny doubles, row-major in j (mass added per step; negative = sink), kept
 * in the workspace in the lattice compute type.  NULL clears it.  LBIB_E_STATE
 * when the context was created with node_sources 0.  Synchronises the
 * context stream. */
int lbib_set_node_sources(lbib_ctx* ctx, const double* S);

/* Choose how many lattice nodes one thread of the lattice update handles.
 * 2 lets FP16 storage update two adjacent nodes per thread, moving every
 * population as one 32-bit word of two halves, whenever the lattice width nx
 * is even; 4 updates four adjacent nodes per thread (one 64-bit word of four
 * halves per population) when nx is a multiple of four, else two; 1 forces
 * one node per thread; 0 (the default) is 2.  FP32 and FP64 storage always use
 * one node per thread.  All give the same arithmetic (the collision of
 * Sec. 6.1, Eq. bgkequation, node by node); the setting exists to compare and
 * time them.  LBIB_E_PARAM for other values.  Waits for the context stream
 * when the choice changes. */
int lbib_set_lattice_variant(lbib_ctx* ctx, int32_t nodes_per_thread);

/* Update the per-cell pressure and source flags of the current cells (the
 * inputs a host-side biology step changes between time steps).  Either
 * pointer may be NULL to keep that array.  The arrays are copied into a
 * pinned staging buffer owned by the context and uploaded asynchronously on
 * the context stream, ordered before the next step; the caller may reuse
 * them as soon as the call returns.  The call waits only for the previous
 * call's upload to have left the staging buffer. */
int lbib_set_cell_params(lbib_ctx* ctx, const double* pressure, const uint8_t* src_flag);

/* Set the populations of species s to the rest equilibrium g_q = w_q phi of
 * the host field phi (nx*ny doubles). */
int lbib_set_species(lbib_ctx* ctx, int32_t s, const double* phi);

/* Advance n_steps coupled time steps (Fig. 1): labels and vertex forces
 * from X^n, spreading, one fused lattice update (stream, moments with the
 * half-force velocity, BGK collision with the body force, all species with
 * the same velocity and their reactions), interpolation of u^n and
 * X^{n+1} = X^n + U^n.  Asynchronous on the context stream.  A non-finite
 * density or velocity is reported by the next lbib_get_fields() as
 * LBIB_E_NONFINITE. */
int lbib_step(lbib_ctx* ctx, int32_t n_steps);

/* Advance n_steps coupled steps exactly like lbib_step() (the same kernels,
 * the same arithmetic and the same state afterwards) without the output
 * work of the last step: no step writes the density, velocity, species,
 * label, force or vertex-force output planes, so every step is an ordinary
 * one and all but at most one are replayed from CUDA graphs.  Afterwards
 * lbib_get_fields() serves LBIB_X and LBIB_AREA; the other fields need an
 * lbib_step() call first (LBIB_E_STATE).  With cell junctions this is
 * lbib_step().  Asynchronous on the context stream. */
int lbib_advance(lbib_ctx* ctx, int32_t n_steps);

/* Copy fields of the last completed step to host buffers (doubles unless
 * stated), synchronising the stream.  `which` is a mask of LBIB_RHO (rho,
 * nx*ny), LBIB_U (ux, uy), LBIB_PHI (phi, n_species*nx*ny), LBIB_X (xy,
 * 2*V, the current vertex positions), LBIB_AREA (area, n_cells, FP64
 * shoelace of the current polygons), LBIB_ID (id, nx*ny int32: 0 outside,
 * c+1 for the lowest cell c containing the node in the last step), LBIB_FORCE (force, 2*nx*ny
 * interleaved fx, fy spread in the last step) and LBIB_VFORCE (vforce, 2*V
 * vertex forces of the last step).  Lattice fields need at least one step
 * since create, the last one by lbib_step() (else LBIB_E_STATE).  Unused pointers may be NULL. */
int lbib_get_fields(lbib_ctx* ctx, uint32_t which, double* rho, double* ux, double* uy,
                    double* phi, double* xy, double* area, int32_t* id, double* force,
                    double* vforce);

/* Asynchronous readback of the cell outputs for a pipelined host loop: the
 * current vertex positions (LBIB_X: xy, 2*V doubles) and/or the FP64 cell
 * areas (LBIB_AREA: area, n_cells) are copied to the host buffers on a copy
 * stream of the context, after the work enqueued so far on the context
 * stream, and the call returns at once.  The steps enqueued afterwards run
 * beside the copies (the first vertex move of lbib_advance() waits for them;
 * lbib_step(), lbib_set_cells(), lbib_set_state() and lbib_get_fields()
 * wait before they start); the buffers must stay valid until
 * lbib_wait_readback() returns, and should be pinned for the copy to overlap.
 * One readback is outstanding at a time: a second call first waits for the
 * previous one and returns its status if that failed.  LBIB_E_PARAM for
 * other bits in `which` or a NULL buffer that is needed.
 * lbib_wait_readback() waits for the outstanding readback (LBIB_OK when
 * there is none) and reports the device diagnostics read with it, as
 * lbib_get_fields() does (LBIB_E_NONFINITE, LBIB_E_CHECK). */
int lbib_get_cells_async(lbib_ctx* ctx, uint32_t which, double* xy, double* area);
int lbib_wait_readback(lbib_ctx* ctx);

/* FP64 conservation sums of the last step's fields (the per-cell and global
 * budgets beside the per-cell area of Sec. 3.3, computeAreas), computed on
 * the device from the output of the last lbib_step() (LBIB_E_STATE after
 * lbib_advance() or before any step) and copied to host buffers;
 * synchronises the stream:
 *   global_sums  3 + n_species doubles: sum rho, sum rho ux, sum rho uy and
 *                sum phi_s over every node (rho u as in LBIB_U: with Guo
 *                forcing it includes half the node's force)
 *   cell_sums    may be NULL, n_cells x (1 + n_species) doubles, row c: sum
 *                rho and sum phi_s over the nodes whose label is cell c (the
 *                lowest cell containing the node, as LBIB_ID)
 *   nonfinite    may be NULL: the number of nodes with a non-finite or
 *                non-positive density or a non-finite velocity or
 *                concentration
 * Accumulated in FP64 (atomic order not fixed: sums agree to rounding). */
int lbib_get_sums(lbib_ctx* ctx, double* global_sums, double* cell_sums, uint32_t* nonfinite);

/* Run n_steps coupled steps like lbib_step(), launching each kernel
 * directly (no graph) with CUDA events recorded on the context stream around
 * every launch, and return the summed device time in milliseconds of the
 * lattice-update launches in ms_out[0] and of the immersed-boundary launches
 * in ms_out[1] (host array of 2; with cell junctions the partner renewals
 * count as immersed-boundary time).  Synchronises the stream. */
int lbib_step_profiled(lbib_ctx* ctx, int32_t n_steps, double* ms_out);

/* Number of vertices and cells currently loaded. */
int lbib_get_sizes(const lbib_ctx* ctx, int32_t* n_vertices, int32_t* n_cells);

/* Raw state snapshot (populations, vertices, cell data) for resume
 * (Sec. 3.1: solver states can be saved and reloaded).  lbib_state_size()
 * gives the byte count; get copies device state to `host`, set restores it
 * into a context created with the same parameters and capacities. */
int lbib_state_size(const lbib_ctx* ctx, uint64_t* bytes_out);
int lbib_get_state(lbib_ctx* ctx, void* host, uint64_t bytes);
int lbib_set_state(lbib_ctx* ctx, const void* host, uint64_t bytes);

/* Label lattice nodes by cell (Fig. 2: the domainID of the lattice nodes is
 * set from the polygons), on the device, without a context.  A node belongs to
 * a cell when its centre is inside the polygon by the crossing-number rule,
 * half-open in y; on overlap the lower cell index is the node's label and
 * the node carries the source flags of every cell containing it.
 *   nx, ny, bc_y              lattice (bc_y 1: rows outside [0, ny) dropped)
 *   n_cells, d_cell_off, d_xy, d_src_flag   device arrays as lbib_set_cells()
 *   d_id       out, nx*ny int32 (dense, row-major): 0 outside, c+1 in cell c
 *   d_src      out (may be NULL), nx*ny bytes: OR of the src_flag of the cells
 *              containing the node
 *   cuda_stream  stream to enqueue on (asynchronous)
 * Returns LBIB_OK, LBIB_E_PARAM or LBIB_E_CUDA (lbib_last_error(NULL)). */
int lbib_label_cells(int32_t nx, int32_t ny, int32_t bc_y, int32_t n_cells,
                     const int32_t* d_cell_off, const double* d_xy, const uint8_t* d_src_flag,
                     int32_t* d_id, uint8_t* d_src, void* cuda_stream);

/* Steady morphogen solve, batched: for each of `batch` independent periodic
 * tissues of nx*ny nodes, the D2Q5 scheme of Sec. 6.1 with u = 0 and the
 * reaction R = src_rate [source node] - decay phi is iterated from its initial
 * state until the residual r = max|phi^{n+1} - phi^n| / max|phi^{n+1}|,
 * evaluated every check_every steps on the last step pair, is <= tol, or
 * max_steps steps have run.  Every tissue stops at its own step count.
 *   d_src       batch*nx*ny bytes (device), bit 0 = source node
 *   D, decay, src_rate   host arrays of batch doubles (D > 0, decay >= 0)
 *   d_phi0      batch*nx*ny floats (device): populations start at the rest
 *               equilibrium g_q = w_q phi0 (a warm start); NULL = cold start
 *               from zero
 *               A warm-started tissue falls back to the cold start (populations
 *               reset to zero, its step count running on) when its residual is
 *               not finite, or when after 64 checks it is not below the residual
 *               of its first check.
 *   d_phi_out   batch*nx*ny floats (device): phi of the final state
 *   steps_out, resid_out  host arrays of batch: steps taken, last residual
 *   fallback_out  host array of batch int32 (may be NULL): 1 where the warm
 *               start was abandoned for the cold one
 *   d_workspace, ws_bytes  device scratch of lbib_steady_workspace_size()
 *               bytes, 256-byte aligned, owned by the caller
 * FP32 storage and arithmetic.  Synchronises the stream.  Returns LBIB_OK,
 * LBIB_E_PARAM, LBIB_E_WORKSPACE or LBIB_E_CUDA. */
int lbib_steady_workspace_size(int32_t nx, int32_t ny, int32_t batch, uint64_t* bytes_out);
int lbib_steady_solve(int32_t nx, int32_t ny, int32_t batch, const uint8_t* d_src,
                      const double* D, const double* decay, const double* src_rate,
                      const float* d_phi0, double tol, int64_t max_steps, int32_t check_every,
                      float* d_phi_out, int64_t* steps_out, double* resid_out,
                      int32_t* fallback_out, void* d_workspace, uint64_t ws_bytes,
                      void* cuda_stream);

/* ---- Ensembles: many independent tissues advanced together -------------
 * An ensemble holds n tissues (each with its own lbib_params -- lattice
 * size, tau, boundary -- and its own cells) in one caller-owned workspace and
 * advances all of them by one persistent cooperative kernel launch per
 * lbib_ensemble_step() call (LBIB_ENS_PERSISTENT: lattice and IB phases
 * separated by grid barriers), or by two launches per step (LBIB_ENS_SPLIT:
 * one lattice launch over every node of every tissue, one IB launch over every
 * cell, ordered by programmatic dependent launches; LBIB_ENS_SPLIT_WIDE: the
 * same with more registers and fewer CTAs per SM for the lattice launch),
 * captured once per step count into a CUDA graph.
 * All tissues use LBIB_FP32 storage and share n_species and forcing.  Each
 * tissue is a context: lbib_ensemble_tissue() returns it for
 * lbib_set_cells(), lbib_get_fields(), lbib_get_state() and the like (do not
 * lbib_destroy() it; lbib_ensemble_destroy() releases all).
 *   lbib_ensemble_workspace_size  bytes for n tissues with the given params
 *                                 and vertex / cell capacities (arrays of n)
 *   lbib_ensemble_create          bind a 256-byte aligned device workspace
 *                                 and a stream; tissues start at rest
 *   lbib_ensemble_step            n_steps of every tissue (asynchronous):
 *                                 the step sequence of lbib_step()
 *   lbib_ensemble_status          synchronise; LBIB_E_TIMEOUT if a grid
 *                                 barrier of the persistent launch waited
 *                                 more than about one second (the launch
 *                                 then ended early and the tissues' state is
 *                                 undefined); the barrier state is reset
 *   lbib_ensemble_config          set the lattice work item (nodes_per_item,
 *                                 a multiple of 256; <= 0 keeps it) and CTAs
 *                                 per SM (0 = as many as fit; < 0 keeps it);
 *                                 reports whether the graph path is in use
 *                                 and the grid size
 *   lbib_ensemble_schedule        set the schedule (LBIB_ENS_PERSISTENT,
 *                                 LBIB_ENS_SPLIT or LBIB_ENS_SPLIT_WIDE; < 0
 *                                 keeps it); schedule_out
 *                                 (may be NULL) receives the one in use;
 *                                 LBIB_E_PARAM for another value
 *   lbib_ensemble_tune            time every (nodes_per_item in 256/512/1024/2048/4096)
 *                                 x (the two split schedules, and the persistent
 *                                 kernel at each CTAs per SM) candidate over
 *                                 trial_steps steps (which advances the
 *                                 tissues), keep the fastest;
 *                                 config_out[2] = {nodes_per_item, the
 *                                 persistent kernel's best CTAs per SM},
 *                                 ms_out = ms per step; the schedule chosen
 *                                 is read with lbib_ensemble_schedule()
 *   lbib_ensemble_selftest_timeout  run one grid barrier that cannot
 *                                 complete, to check that the bounded wait
 *                                 ends (seconds_out) and is reported as
 *                                 LBIB_E_TIMEOUT
 * The paper runs one tissue per process (Sec. 3.4); the ensemble is the
 * parameter-sweep form of the same step. */
typedef struct lbib_ensemble lbib_ensemble;
#define LBIB_ENS_PERSISTENT 0
#define LBIB_ENS_SPLIT 1
#define LBIB_ENS_SPLIT_WIDE 2
int lbib_ensemble_workspace_size(int32_t n, const lbib_params* params,
                                 const int32_t* max_vertices, const int32_t* max_cells,
                                 uint64_t* bytes_out);
int lbib_ensemble_create(int32_t n, const lbib_params* params, const int32_t* max_vertices,
                         const int32_t* max_cells, void* d_workspace, uint64_t bytes,
                         void* cuda_stream, lbib_ensemble** out);
lbib_ctx* lbib_ensemble_tissue(lbib_ensemble* ens, int32_t t);
int lbib_ensemble_step(lbib_ensemble* ens, int32_t n_steps);
int lbib_ensemble_status(lbib_ensemble* ens);
int lbib_ensemble_config(lbib_ensemble* ens, int32_t nodes_per_item, int32_t blocks_per_sm,
                         int32_t* graph_out, int32_t* grid_out);
int lbib_ensemble_schedule(lbib_ensemble* ens, int32_t schedule, int32_t* schedule_out);
int lbib_ensemble_tune(lbib_ensemble* ens, int32_t trial_steps, int32_t* config_out,
                       double* ms_out);
int lbib_ensemble_selftest_timeout(lbib_ensemble* ens, double* seconds_out);
void lbib_ensemble_destroy(lbib_ensemble* ens);
const char* lbib_ensemble_last_error(const lbib_ensemble* ens);

/* ---- Neural operator: learned warm start of the steady morphogen solve ----
 * The paper has no network; this is the learned part the measured method adds
 * in front of lbib_steady_solve().  A six-level convolutional U-Net maps, per
 * tissue, [cell mask, source mask, (D - 0.125)/0.075, log10(decay) + 3] on an
 * H x W lattice to y, and predicts phi = y * src_rate / decay; it is trained
 * on targets phi * decay / src_rate with mean squared error and Adam
 * (0.9, 0.999, 1e-8).  Levels have 32, 48, 64, 96, 128, 192 channels; each is
 * conv3x3-ReLU-conv3x3-ReLU, joined by 2x2 average pooling; the decoder
 * convolves [skip, upsample2(deeper)]; a final conv3x3 gives one channel.
 * Weights are FP32 masters with BF16 copies; activations BF16; every
 * convolution runs on the tensor cores with FP32 accumulation.
 *   lbib_nop_workspace_size / lbib_nop_create  up to `batch` tissues of
 *              H x W (multiples of 32) per call; caller-owned 256-byte
 *              aligned device workspace; parameters start at zero
 *   lbib_nop_num_params   parameter count in the canonical flat layout:
 *              per layer (in order) weights (3, 3, Ci, Co) then bias (Co)
 *   lbib_nop_layers       layer count and (Ci, Co) pairs of that layout
 *   lbib_nop_set_params / get_params / get_grads  host FP32 vectors in that
 *              layout (set also resets the Adam state)
 *   lbib_nop_forward      phi prediction (d_phi, n*H*W floats) from device
 *              masks (n*H*W bytes, nonzero = inside) and host per-tissue D,
 *              decay, src_rate (n doubles each)
 *   lbib_nop_train_step   forward, loss, backward; with update != 0 also one
 *              Adam step of learning rate lr; loss_out = the batch loss
 * Synchronising calls.  Errors as elsewhere; lbib_nop_last_error(). */
typedef struct lbib_nop lbib_nop;
int lbib_nop_workspace_size(int32_t batch, int32_t H, int32_t W, uint64_t* bytes_out);
int lbib_nop_create(int32_t batch, int32_t H, int32_t W, void* d_workspace, uint64_t bytes,
                    void* cuda_stream, lbib_nop** out);
int lbib_nop_num_params(const lbib_nop* nop, int64_t* count);
int lbib_nop_layers(const lbib_nop* nop, int32_t* n_layers, int32_t* ci_co);
int lbib_nop_set_params(lbib_nop* nop, const float* host, int64_t count);
int lbib_nop_get_params(lbib_nop* nop, float* host, int64_t count);
int lbib_nop_get_grads(lbib_nop* nop, float* host, int64_t count);
int lbib_nop_forward(lbib_nop* nop, int32_t n, const uint8_t* d_mask, const uint8_t* d_src,
                     const double* D, const double* decay, const double* src_rate, float* d_phi);
int lbib_nop_train_step(lbib_nop* nop, int32_t n, const uint8_t* d_mask, const uint8_t* d_src,
                        const double* D, const double* decay, const double* src_rate,
                        const float* d_phi_target, double lr, int32_t update,
                        double* loss_out);
void lbib_nop_destroy(lbib_nop* nop);
const char* lbib_nop_last_error(const lbib_nop* nop);

/* Single layers of the network (device pointers, asynchronous on the stream):
 *   lbib_nn_conv3x3        out = conv3x3(in) + bias (ReLU if relu), zero
 *                          padding; input = [in1 (N,H,W,C1), upsample2(in2)
 *                          (N,H/2,W/2,C2)] concatenated on channels (C2 may be
 *                          0); BF16 NHWC in, weights d_wf BF16 (9, Co, C1+C2),
 *                          bias FP32 (Co) or NULL, out BF16 or FP32 (out_f32)
 *                          (N,H,W,Co); C1, C2 multiples of 16, Co even
 *   lbib_nn_conv3x3_wgrad  d_dw (9, C1+C2, Co) += sum over pixels of
 *                          in(shifted) x d_g, d_db (Co) += sum of d_g (FP32,
 *                          accumulated: zero them first); Co multiple of 8
 *   lbib_nn_weight_copies  from FP32 (3,3,Ci,Co) weights the BF16 forward
 *                          copy (9, Cop, Cip) and the tap-flipped data-gradient
 *                          copy (9, Cip, Cop), zero padded to Cip, Cop */
int lbib_nn_conv3x3(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                    const void* d_in1, const void* d_in2, const void* d_wf, const float* d_bias,
                    void* d_out, int32_t relu, int32_t out_f32, void* cuda_stream);
int lbib_nn_conv3x3_wgrad(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                          const void* d_in1, const void* d_in2, const void* d_g, float* d_dw,
                          float* d_db, void* cuda_stream);
int lbib_nn_weight_copies(int32_t Ci, int32_t Co, int32_t Cip, int32_t Cop, const float* d_w,
                          void* d_wf, void* d_wd, void* cuda_stream);

/* The same 3x3 convolution on the fifth-generation tensor cores (tcgen05.mma
 * with the FP32 accumulator in tensor memory, operands staged by the tensor
 * memory accelerator); the network's training and inference use it for the
 * levels where it is the faster kernel:
 *   lbib_nn_conv3x3_tc_supported  1 when the shape is supported: W <= 128 or
 *                          a multiple of 128; C1 >= 16, C1 and C2 multiples
 *                          of 16, and C1 a multiple of 32 when C1 + C2 is
 *                          (the chunk width); H and W even when C2 > 0;
 *                          Co >= 1
 *   lbib_nn_tile_weights_tc  the forward weights d_wf (9, Co, Ci) (as
 *                          lbib_nn_weight_copies makes them) rearranged into
 *                          d_wt, the order and the swizzled layout the
 *                          kernel's bulk copies load (*elems_out bf16
 *                          elements; d_wt NULL: size only)
 *   lbib_nn_conv3x3_tc     out = conv3x3([in1, upsample2(in2)]) + bias (ReLU
 *                          if relu) as lbib_nn_conv3x3, with the tiled weights;
 *                          d_in1, d_in2, d_wt, d_out 16-byte aligned; d_err a device
 *                          word the caller zeroes: nonzero afterwards when a
 *                          bounded wait of the kernel ran out (the output is
 *                          then undefined)
 * The paper has no network; these calls belong to the learned warm start. */
int lbib_nn_conv3x3_tc_supported(int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co);
int lbib_nn_tile_weights_tc(int32_t Ci, int32_t Co, const void* d_wf, void* d_wt,
                            uint64_t* elems_out, void* cuda_stream);
int lbib_nn_conv3x3_tc(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                       const void* d_in1, const void* d_in2, const void* d_wt, const float* d_bias,
                       void* d_out, int32_t relu, int32_t out_f32, uint32_t* d_err,
                       void* cuda_stream);

/* The weight gradient on the tensor cores (tcgen05.mma with MN-major operands:
 * the pixels are the contraction, the input channels of three tap shifts the
 * M rows, the output channels the N rows; FP32 accumulators in tensor memory,
 * added to d_dw with FP32 reductions):
 *   lbib_nn_conv3x3_wgrad_tc_supported  1 when the shape is supported: W from 16
 *                          to 128 in multiples of 16, or a multiple of 128;
 *                          C1 >= 16, C1 and C2 multiples of 16, C1 + C2 <= 384;
 *                          Co a multiple of 16; H and W even when C2 > 0
 *   lbib_nn_conv3x3_wgrad_tc  as lbib_nn_conv3x3_wgrad (d_dw (9, C1+C2, Co) and
 *                          d_db (Co, or NULL) accumulated: zero them first);
 *                          d_in1, d_in2, d_g, d_dw 16-byte aligned; d_err as for
 *                          lbib_nn_conv3x3_tc */
int lbib_nn_conv3x3_wgrad_tc_supported(int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co);
int lbib_nn_conv3x3_wgrad_tc(int32_t N, int32_t H, int32_t W, int32_t C1, int32_t C2, int32_t Co,
                             const void* d_in1, const void* d_in2, const void* d_g, float* d_dw,
                             float* d_db, uint32_t* d_err, void* cuda_stream);

/* Coupled steps without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate device memory while
 * they run -- code inside a framework whose memory pool owns the device, or
 * plug-ins that must keep the device footprint fixed after start-up.  It runs
 * the kernels of lbib_step() on state the caller already owns and calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *
 * The intermediate planes (second population buffer, spread force, source
 * bits, velocity, diagnostic words) live in one static device array of 4 MiB
 * inside the library; every GPU that loads the library holds it until the
 * process exits.  Lattices whose planes do not fit are rejected with
 * LBIB_E_WORKSPACE (with FP64 storage and one species, 64x64 needs about
 * 0.6 MiB and 128x128 about 2.4 MiB; 192x192 does not fit).
 * All calls share the array: calls that overlap on the GPU (two streams, two
 * host threads) race and give wrong results, so serialise them.  Each call
 * resets the planes that must start empty.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current.  The call reads the diagnostic words back and synchronises
 * `cuda_stream` before it returns, so that stream must not be capturing a
 * graph when it is called.
 *
 * Arguments (device pointers, on the current device):
 *   params      as for lbib_create() (the same checks); params->precision
 *               selects the storage; confined species, junctions, mass
 *               sources, pressure nodes and node sources are refused
 *               (LBIB_E_PARAM: they need a context's planes)
 *   n_cells, d_cell_off, d_xy (in/out, 2*V), d_rest_len, d_k_spring (V),
 *               d_pressure (n_cells), d_src_flag (n_cells): as lbib_set_cells()
 *               but already on the device and complete (no NULL defaults);
 *               the offsets are not read on the host, so a cell with fewer
 *               than 3 or more than 1024 vertices is skipped on the device
 *               and reported as LBIB_E_NONFINITE (geometry flag)
 *   d_f         9 population planes, d_g 5*n_species planes (in/out), in the
 *               library's storage layout: element bytes b = 8 / 4 / 2 for
 *               FP64 / FP32 / FP16, row pitch = nx rounded up to a multiple
 *               of 64 elements, plane stride = pitch*ny + 1536/b elements,
 *               values stored as the deviations f - w rho0 (FP16: divided by
 *               w sigma) -- the population section of lbib_get_state(); all
 *               zero bytes is the rest state
 *   alignment   d_f, d_g and d_xy 16 bytes; d_rest_len, d_k_spring,
 *               d_pressure 8 bytes; d_cell_off 4 bytes (else LBIB_E_PARAM)
 *   n_steps     steps to advance; the result is always left in d_f, d_g
 *   cuda_stream cudaStream_t as void* (NULL = legacy default stream)
 * Returns LBIB_OK, LBIB_E_PARAM, LBIB_E_WORKSPACE (lattice too large for the
 * static array), LBIB_E_NONFINITE or LBIB_E_CUDA; lbib_last_error(NULL) gives
 * the reason. */
int lbib_step_noalloc(const lbib_params* params, int32_t n_cells, const int32_t* d_cell_off,
                      double* d_xy, const double* d_rest_len, const double* d_k_spring,
                      const double* d_pressure, const uint8_t* d_src_flag, void* d_f,
                      void* d_g, int32_t n_steps, void* cuda_stream);

/* Release the host header (the workspace stays the caller's). */
void lbib_destroy(lbib_ctx* ctx);

/* One-line description of the last error on ctx (or of the last failed
 * lbib_create when ctx is NULL). */
const char* lbib_last_error(const lbib_ctx* ctx);

/* Static name of a status code. */
const char* lbib_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBIB_H */
