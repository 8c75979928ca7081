// lbib.cu -- host engine and C ABI of the coupled LB-IB library.
//
// The context binds a caller-owned device workspace (layout below), keeps
// the tau-derived coefficients, and sequences the kernels of a time step on
// the caller's stream:
//
//   step n:  [IB prep  X^n -> labels, F^n, spread]      (ib.cu)
//            [lattice  stream, collide fluid + species] (lattice.cu)
//            [IB move  U^n = interp(u^n), X^{n+1}]       (ib.cu)
//
// Between two steps the move of step n and the prep of step n+1 are one
// launch, so a step costs two launches.  A chunk of two steps (one full A/B
// buffer cycle) is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbib_ctx.cuh"
#include "lbib_internal.cuh"

namespace lbib {

static uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

bool make_layout(const lbib_params& p, int max_vertices, int max_cells, Layout* L) {
    if (p.nx < 8 || p.ny < 8 || p.nx > (1 << 20) || p.ny > (1 << 20)) return false;
    if (p.precision < LBIB_FP64 || p.precision > LBIB_FP16) return false;
    if (p.n_species < 0 || p.n_species > kMaxSpecies) return false;
    if (max_vertices < 0 || max_cells < 0 || max_cells > (1 << 27)) return false;
    Layout l;
    l.es = p.precision == LBIB_FP64 ? 8 : (p.precision == LBIB_FP32 ? 4 : 2);
    l.cs = p.precision == LBIB_FP64 ? 8 : 4;
    l.pitch = (int64_t)align_up((uint64_t)p.nx, 64);
    // planes are padded by 1.5 KiB (six 256-byte blocks) so that the 9 + 5S
    // streams of one node do not sit at a power-of-two distance from each other
    l.plane = l.pitch * p.ny + 1536 / l.es;
    // the kernels index within a plane with 32-bit integers
    if (l.plane > (int64_t)0x7FFFFFFF) return false;
    const uint64_t P = (uint64_t)l.plane;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    l.f[0] = take(9 * P * l.es);
    l.f[1] = take(9 * P * l.es);
    l.g[0] = take((uint64_t)5 * p.n_species * P * l.es);
    l.g[1] = take((uint64_t)5 * p.n_species * P * l.es);
    l.force = take(2 * P * l.cs);
    l.u = take(2 * P * l.cs);
    l.rho = take(P * l.cs);
    l.phi = take((uint64_t)p.n_species * P * l.cs);
    l.id = take(P * 4);
    l.id_out = take(P * 4);
    l.fmask = take((uint64_t)mask_words(l.plane) * 4);
    l.lmask = take((uint64_t)mask_words(l.plane) * 4);
    l.src = take(align_up(P, 8));  // one byte per node
    l.smask = take((uint64_t)mask_words(l.plane) * 4);
    l.force_out = take(2 * P * l.cs);
    if (p.noflux_mask) l.dom = take(P * 4);
    if (p.noflux_mask && p.noflux_scheme == LBIB_NOFLUX_CLOSURE) {
        l.ncode = take(P * 2);
        l.mom[0] = take((uint64_t)3 * p.n_species * P * l.cs);
        l.mom[1] = take((uint64_t)3 * p.n_species * P * l.cs);
    }
    if (p.mass_sources && max_cells > 0) {
        l.mrate = take((uint64_t)max_cells * 8);
        l.marea = take((uint64_t)max_cells * 8);
        l.msrc = take((uint64_t)max_cells * 8);
    }
    if (p.pressure_nodes) l.pnode = take(align_up(P, 8));
    if (p.node_sources) l.nsrc = take(P * l.cs);
    if (p.junction_period > 0 && max_cells > 0) {
        // bins at least l_max wide (with a margin against rounding at their
        // edges); wider where they would outnumber the vertices by far
        const double bw = p.junction_lmax * 1.0001;
        l.jnbx = std::max(1, (int)std::floor(p.nx / bw));
        l.jnby = std::max(1, (int)std::floor(p.ny / bw));
        const int64_t cap = std::min<int64_t>(1 << 22, std::max<int64_t>(4096, 4 * (int64_t)max_vertices));
        while ((int64_t)l.jnbx * l.jnby > cap) {
            if (l.jnbx >= l.jnby)
                l.jnbx = (l.jnbx + 1) / 2;
            else
                l.jnby = (l.jnby + 1) / 2;
        }
        const uint64_t nb = (uint64_t)l.jnbx * l.jnby;
        l.jpartner = take((uint64_t)max_vertices * 4);
        l.jcell = take((uint64_t)max_vertices * 4);
        l.jcnt = take(nb * 4);
        l.jstart = take((nb + 1) * 4);
        l.jvbin = take((uint64_t)max_vertices * 4);
        l.jent = take((uint64_t)max_vertices * sizeof(JunctionEntry));
    }
    const uint64_t V = (uint64_t)max_vertices, C = (uint64_t)max_cells;
    l.xy = take(V * 16);
    l.L0 = take(V * 8);
    l.k = take(V * 8);
    l.vforce = take(V * 16);
    l.vbase = take(V * 8);
    l.vfrac = take(V * 8);
    l.off = take((C + 1) * 4);
    l.pres = take(C * 8);
    l.srcf = take(C);
    l.area = take(C * 8);
    l.sums_bytes = (uint64_t)(4 + kMaxSpecies + C * (1 + kMaxSpecies)) * 8 + 16;
    l.sums = take(l.sums_bytes);
    l.diag = take(kDiagWords * 4);
    l.total = o;
    *L = l;
    return true;
}

}  // namespace lbib

using namespace lbib;


static thread_local std::string g_create_err;

static int fail(lbib_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

static int cuda_fail(lbib_ctx* c, cudaError_t e, const char* where) {
    return fail(c, LBIB_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static int check_params(const lbib_params* p, std::string* why) {
    if (!p) { *why = "params is NULL"; return LBIB_E_PARAM; }
    if (p->nx < 8 || p->ny < 8) { *why = "nx and ny must be >= 8"; return LBIB_E_PARAM; }
    if ((int64_t)p->nx * p->ny > ((int64_t)1 << 34)) { *why = "lattice too large"; return LBIB_E_PARAM; }
    if (p->bc_y != 0 && p->bc_y != 1) { *why = "bc_y must be 0 or 1"; return LBIB_E_PARAM; }
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { *why = "tau must be > 1/2"; return LBIB_E_PARAM; }
    if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) { *why = "rho0 must be > 0"; return LBIB_E_PARAM; }
    if (p->n_species < 0 || p->n_species > 4) { *why = "n_species must be 0..4"; return LBIB_E_PARAM; }
    for (int s = 0; s < p->n_species; ++s)
        if (!(p->D[s] > 0.0) || !std::isfinite(p->D[s])) { *why = "D must be > 0"; return LBIB_E_PARAM; }
    if (p->forcing != LBIB_GUO && p->forcing != LBIB_HE_PAPER) { *why = "unknown forcing"; return LBIB_E_PARAM; }
    if (p->precision < LBIB_FP64 || p->precision > LBIB_FP16) { *why = "unknown precision"; return LBIB_E_PARAM; }
    if (p->fp16_scale < 0 || p->fp16_scale_species < 0) { *why = "fp16 scales must be >= 0"; return LBIB_E_PARAM; }
    if (p->reaction != LBIB_REACT_LINEAR && p->reaction != LBIB_REACT_SCHNAKENBERG) {
        *why = "unknown reaction model"; return LBIB_E_PARAM;
    }
    if (p->reaction == LBIB_REACT_SCHNAKENBERG &&
        (p->n_species < 2 || !std::isfinite(p->schnak[0]) || !std::isfinite(p->schnak[1]) ||
         !std::isfinite(p->schnak[2]))) {
        *why = "the Schnakenberg reaction needs two species and finite gamma, a, b";
        return LBIB_E_PARAM;
    }
    if (p->noflux_mask < 0 || p->noflux_mask >= (1 << p->n_species)) {
        *why = "noflux_mask names a species that does not exist"; return LBIB_E_PARAM;
    }
    if (p->noflux_scheme != LBIB_NOFLUX_CLOSURE && p->noflux_scheme != LBIB_NOFLUX_BOUNCEBACK) {
        *why = "noflux_scheme must be LBIB_NOFLUX_CLOSURE or LBIB_NOFLUX_BOUNCEBACK";
        return LBIB_E_PARAM;
    }
    if (p->junction_period < 0 ||
        (p->junction_period > 0 &&
         (!(p->junction_lmax > 0.0) || !std::isfinite(p->junction_lmax) ||
          !std::isfinite(p->junction_k) || !(p->junction_l0 >= 0.0) ||
          p->junction_lmax * 3.0 > std::min(p->nx, p->ny)))) {
        *why = "junctions need period >= 0, 0 < l_max <= min(nx, ny)/3, finite k, l0 >= 0";
        return LBIB_E_PARAM;
    }
    if ((p->mass_sources != 0 && p->mass_sources != 1) || !std::isfinite(p->mass_alpha)) {
        *why = "mass_sources must be 0 or 1 and mass_alpha finite"; return LBIB_E_PARAM;
    }
    if ((p->pressure_nodes != 0 && p->pressure_nodes != 1) ||
        (p->pressure_nodes && (!(p->pressure_rho > 0.0) || !std::isfinite(p->pressure_rho)))) {
        *why = "pressure_nodes must be 0 or 1 and pressure_rho finite and > 0";
        return LBIB_E_PARAM;
    }
    if (p->node_sources != 0 && p->node_sources != 1) {
        *why = "node_sources must be 0 or 1"; return LBIB_E_PARAM;
    }
    return LBIB_OK;
}

template <typename C>
static void fill_coefs(const lbib_params& p, Coefs<C>* k) {
    std::memset(k, 0, sizeof(*k));
    k->rho0 = (C)p.rho0;
    k->omega = (C)(1.0 / p.tau);
    k->omc = (C)(1.0 - 1.0 / p.tau);
    k->pref = (C)(1.0 - 0.5 / p.tau);
    k->bfx = (C)p.body_force[0];
    k->bfy = (C)p.body_force[1];
    for (int s = 0; s < kMaxSpecies; ++s) {
        double tauD = 3.0 * p.D[s] + 0.5;
        k->omegaD[s] = (C)(s < p.n_species ? 1.0 / tauD : 0.0);
        k->omcD[s] = (C)(s < p.n_species ? 1.0 - 1.0 / tauD : 1.0);
        k->srate[s] = (C)p.src_rate[s];
        for (int b = 0; b < kMaxSpecies; ++b)
            k->K[s][b] = (C)(p.react[s][b] - (s == b ? p.decay[s] : 0.0));
    }
    k->react_model = p.reaction;
    k->sgamma = (C)p.schnak[0];
    k->sa = (C)p.schnak[1];
    k->sb = (C)p.schnak[2];
    k->prho = (C)(p.pressure_nodes ? p.pressure_rho : p.rho0);
    const double sf = p.fp16_scale > 0 ? p.fp16_scale : std::ldexp(1.0, -10);
    const double sg = p.fp16_scale_species > 0 ? p.fp16_scale_species : std::ldexp(1.0, -8);
    const bool scaled = p.precision == LBIB_FP16;
    k->isig = (C)(scaled ? 1.0 / sf : 1.0);
    k->isig_g = (C)(scaled ? 1.0 / sg : 1.0);
    exact_sum_weights<C>(k->w9c, k->w5c);
    for (int q = 0; q < 9; ++q) {
        const double wq = (double)k->w9c[q == 0 ? 0 : (q < 5 ? 1 : 2)];
        k->fscale[q] = (C)(scaled ? wq * sf : 1.0);
        k->finv[q] = (C)(scaled ? 1.0 / (wq * sf) : 1.0);
    }
    for (int q = 0; q < 5; ++q) {
        const double wq = (double)k->w5c[q == 0 ? 0 : 1];
        k->gscale[q] = (C)(scaled ? wq * sg : 1.0);
        k->ginv[q] = (C)(scaled ? 1.0 / (wq * sg) : 1.0);
    }
}

namespace lbib {
void fill_coefs_public(const lbib_params& p, Coefs<double>* k) { fill_coefs(p, k); }
void fill_coefs_public(const lbib_params& p, Coefs<float>* k) { fill_coefs(p, k); }
int check_params_public(const lbib_params* p, std::string* why) { return check_params(p, why); }
int set_thread_error(int code, const std::string& msg) {
    g_create_err = msg;
    return code;
}
}  // namespace lbib

static const void* coefs_of(const lbib_ctx* c) {
    return c->p.precision == LBIB_FP64 ? (const void*)&c->kd : (const void*)&c->kf;
}

static LatticeArgs lattice_args(lbib_ctx* c, int src_buf, bool out) {
    LatticeArgs a;
    std::memset(&a, 0, sizeof(a));
    const Layout& L = c->L;
    a.fsrc = c->ws + L.f[src_buf];
    a.fdst = c->ws + L.f[1 - src_buf];
    a.gsrc = c->ws + L.g[src_buf];
    a.gdst = c->ws + L.g[1 - src_buf];
    a.force = c->ws + L.force;
    a.id = c->at<uint32_t>(L.id);
    a.u = c->ws + L.u;
    a.rho = c->ws + L.rho;
    a.phi = c->ws + L.phi;
    a.id_out = c->at<uint32_t>(L.id_out);
    a.force_out = c->ws + L.force_out;
    a.diag = c->at<uint32_t>(L.diag);
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.pitch = L.pitch;
    a.plane = L.plane;
    a.out = out ? 1 : 0;
    a.ib = c->nC > 0 ? 1 : 0;
    a.l2_first = c->l2_first ? 1 : 0;
    if (c->p.noflux_mask) {
        a.dom = c->at<int32_t>(L.dom);
        a.noflux = c->p.noflux_mask;
        if (L.ncode) {  // the closure: moments by the parity of the population buffers
            a.ncode = c->at<uint16_t>(L.ncode);
            a.mom_in = c->ws + L.mom[src_buf];
            a.mom_out = c->ws + L.mom[1 - src_buf];
        }
    }
    a.fmask = c->at<uint32_t>(L.fmask);
    a.lmask = c->at<uint32_t>(L.lmask);
    a.src = c->at<uint8_t>(L.src);
    a.smask = c->at<uint32_t>(L.smask);
    if (c->p.mass_sources && c->nC > 0) a.msrc = c->ws + L.msrc;
    if (c->p.pressure_nodes) a.pnode = c->at<uint8_t>(L.pnode);
    if (c->p.node_sources) a.nsrc = c->ws + L.nsrc;
    return a;
}

// out_next: the prep is for the output step (vertex forces and labels are
// written for the caller)
static IBArgs ib_args(lbib_ctx* c, bool move, bool prep, bool out_next) {
    IBArgs a;
    std::memset(&a, 0, sizeof(a));
    const Layout& L = c->L;
    if (c->p.junction_period > 0 && prep && !move && L.jpartner) {
        // the partners' positions are read while no vertex moves
        a.jpartner = c->at<int32_t>(L.jpartner);
        a.jk = c->p.junction_k;
        a.jl0 = c->p.junction_l0;
        a.jlmax = c->p.junction_lmax;
    }
    a.xy = c->at<double2>(L.xy);
    a.L0 = c->at<double>(L.L0);
    a.k = c->at<double>(L.k);
    a.off = c->at<int32_t>(L.off);
    a.pres = c->at<double>(L.pres);
    a.srcf = c->at<uint8_t>(L.srcf);
    a.vforce = c->at<double2>(L.vforce);
    a.force = c->ws + L.force;
    a.id = c->at<uint32_t>(L.id);
    a.u = c->ws + L.u;
    a.diag = c->at<uint32_t>(L.diag);
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.bc_y = c->p.bc_y;
    a.n_cells = c->nC;
    a.pitch = L.pitch;
    a.plane = L.plane;
    a.tension = c->p.tension;
    a.do_move = move ? 1 : 0;
    a.do_prep = prep ? 1 : 0;
    a.do_mask = 1;
    a.write_vforce = out_next ? 1 : 0;
    a.do_ids = out_next ? 1 : 0;
    a.do_force = 1;
    a.vbase = c->at<int2>(L.vbase);
    a.vfrac = c->at<float2>(L.vfrac);
    a.fmask = c->at<uint32_t>(L.fmask);
    a.lmask = c->at<uint32_t>(L.lmask);
    a.src = c->at<uint8_t>(L.src);
    a.smask = c->at<uint32_t>(L.smask);
    if (c->p.mass_sources && prep && L.msrc) {
        // S_c for the coming lattice update, at every node labelled c: the
        // labels are needed every step
        a.msrc_out = c->ws + L.msrc;
        a.mrate = c->at<double>(L.mrate);
        a.marea = c->mass_ctrl ? c->at<double>(L.marea) : nullptr;
        a.malpha = c->p.mass_alpha;
        a.do_ids = 1;
    }
    return a;
}

namespace lbib {
LatticeArgs ctx_lattice_args(lbib_ctx* c, int src_buf, bool out) { return lattice_args(c, src_buf, out); }
IBArgs ctx_ib_args(lbib_ctx* c, bool move, bool prep, bool out_next) {
    return ib_args(c, move, prep, out_next);
}
}  // namespace lbib

// pdl: programmatic launch, allowed only when the previous launch on the
// stream is the other kernel of the step (an IB launch before a lattice
// launch and vice versa): each kernel's early loads rely on the launch two
// back having completed, which the other kernel's wait guarantees.
// The no-flux closure reads the species moments of the previous step; after
// create, lbib_set_species, lbib_set_domains or lbib_set_state there is no
// previous step, and the moments of the stored populations stand in.
static cudaError_t ensure_moments(lbib_ctx* c) {
    if (!c->L.ncode || c->mom_valid) return cudaSuccess;
    cudaError_t e = launch_species_moments(c->p.precision, c->p.n_species, c->p.nx, c->p.ny,
                                           c->L.pitch, c->L.plane, c->ws + c->L.g[c->cur],
                                           c->ws + c->L.mom[c->cur], coefs_of(c), c->stream);
    if (e == cudaSuccess) c->mom_valid = true;
    return e;
}

static cudaError_t enqueue_lattice(lbib_ctx* c, int src_buf, bool out, bool pdl = false) {
    NvtxRange nvtx_range("lbib.lattice_update");
    LatticeArgs a = lattice_args(c, src_buf, out);
    return launch_lattice(c->p.precision, c->p.n_species, c->p.bc_y, c->p.forcing, a,
                          coefs_of(c), c->block, c->stream, pdl && c->nC > 0, c->lattice_npt);
}

static cudaError_t enqueue_ib(lbib_ctx* c, bool move, bool prep, bool out_next,
                              bool pdl = false) {
    NvtxRange nvtx_range("lbib.ib_cells");
    if (c->nC == 0) return cudaSuccess;
    return launch_ib(c->p.precision, ib_args(c, move, prep, out_next), c->maxv_cell, c->stream,
                     pdl);
}

static void drop_graphs(lbib_ctx* c) {
    for (int i = 0; i < 2; ++i) {
        if (c->chunk[i]) {
            cudaGraphExecDestroy(c->chunk[i]);
            c->chunk[i] = nullptr;
        }
        if (c->tail[i]) {
            cudaGraphExecDestroy(c->tail[i]);
            c->tail[i] = nullptr;
        }
    }
    c->chunk_nC = -1;
}

// two full steps starting from buffer parity `par`, ending with the prep of
// the following step: [lat(par), ib move+prep, lat(1-par), ib move+prep];
// inside the graph each launch after the first is programmatic
// tail: the second IB launch only moves (no prep for a following step)
static cudaError_t enqueue_chunk(lbib_ctx* c, int par, bool tail = false) {
    cudaError_t e = enqueue_lattice(c, par, false);
    if (e == cudaSuccess) e = enqueue_ib(c, true, true, false, true);
    if (e == cudaSuccess) e = enqueue_lattice(c, 1 - par, false, true);
    if (e == cudaSuccess) e = enqueue_ib(c, true, !tail, false, true);
    return e;
}

static cudaError_t get_chunk_graph(lbib_ctx* c, int par, cudaGraphExec_t* out,
                                   bool tail = false) {
    if (c->chunk_nC != c->nC) drop_graphs(c);
    cudaGraphExec_t* slot = tail ? &c->tail[par] : &c->chunk[par];
    if (!*slot) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        cudaStream_t saved = c->stream;
        c->stream = cap;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_chunk(c, par, tail);
            e = cudaStreamEndCapture(cap, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        c->stream = saved;
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e;
        }
        e = cudaGraphInstantiate(slot, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        c->chunk_nC = c->nC;
    }
    *out = *slot;
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Steps with cell junctions.  The prep of step n needs the positions X^n of
// every cell (the partners of a cell's vertices belong to other cells), so
// the move of step n - 1 and the prep of step n run as separate launches,
// with the renewal of the partners between them when n is a multiple of
// the period.  Launched one by one (no graph): the renewal is decided on the
// host from the step count.
static bool junction_due(const lbib_ctx* c) { return c->nstep % c->p.junction_period == 0; }

static cudaError_t junction_renew(lbib_ctx* c) {
    const Layout& L = c->L;
    JunctionArgs j;
    std::memset(&j, 0, sizeof(j));
    j.xy = c->at<double2>(L.xy);
    j.vcell = c->at<int32_t>(L.jcell);
    j.partner = c->at<int32_t>(L.jpartner);
    j.cnt = c->at<int>(L.jcnt);
    j.start = c->at<int>(L.jstart);
    j.vbin = c->at<int>(L.jvbin);
    j.ent = c->at<JunctionEntry>(L.jent);
    j.nv = c->nV;
    j.nx = c->p.nx;
    j.ny = c->p.ny;
    j.bc_y = c->p.bc_y;
    j.nbx = L.jnbx;
    j.nby = L.jnby;
    j.inv_nx = 1.0 / c->p.nx;
    j.inv_ny = 1.0 / c->p.ny;
    j.inv_wbx = L.jnbx / (double)c->p.nx;
    j.inv_wby = L.jnby / (double)c->p.ny;
    j.lmax = c->p.junction_lmax;
    // FP32 prefilter: the wrapped FP32 coordinates are within n 2^-24 of the
    // exact ones, a folded FP32 difference within 4 n 2^-24 of the exact
    // minimum image, so a candidate at an exact distance below l_max has an
    // FP32 distance below l_max + 6 n 2^-24 (with the norm's rounding inside
    // the 1e-5 relative margin)
    const double eps = 6.0 * std::max(c->p.nx, c->p.ny) * std::ldexp(1.0, -24);
    const double r = (j.lmax + eps) * (1.0 + 1e-5);
    j.fthr = (float)(r * r);
    return launch_junction_renew(j, c->stream);
}

// Steps with cell junctions.  The junction force of a vertex needs the moved
// position of a vertex of another cell, so the move and the next step's prep
// are two launches with the partner renewal between them when it is due.
// `wrap(kind, fn)` runs one enqueue (kind 0 lattice, 1 everything else) and
// returns its status; the profiled step brackets it with events.
// With pdl the lattice update (after the prep) and the move (after the
// update) are programmatic launches: the update's early population loads need
// the previous update finished, which the previous move waited for before the
// prep (an ordinary launch) could start; the move's early loads of the
// vertex bases need the prep finished, which the update waits for before it
// lets the move start.  Preps and renewals stay ordinary launches.
template <class Wrap>
static cudaError_t run_with_junctions(lbib_ctx* c, int n_steps, bool pdl, Wrap&& wrap) {
    cudaError_t e = cudaSuccess;
    if (junction_due(c)) e = wrap(1, [&] { return junction_renew(c); });
    if (e == cudaSuccess) e = wrap(1, [&] { return enqueue_ib(c, false, true, n_steps == 1); });
    for (int i = 0; i < n_steps && e == cudaSuccess; ++i) {
        const bool last = (i == n_steps - 1);
        e = wrap(0, [&] { return enqueue_lattice(c, c->cur, last, pdl); });
        if (e == cudaSuccess) e = wrap(1, [&] { return enqueue_ib(c, true, false, false, pdl); });
        c->cur = 1 - c->cur;
        ++c->nstep;
        if (e == cudaSuccess && !last) {
            if (junction_due(c)) e = wrap(1, [&] { return junction_renew(c); });
            if (e == cudaSuccess)
                e = wrap(1, [&] { return enqueue_ib(c, false, true, i == n_steps - 2); });
        }
    }
    return e;
}

// the cell index of every vertex, for the junction search
static cudaError_t upload_vertex_cells(lbib_ctx* c, int n_cells, const int32_t* cell_off) {
    if (!c->L.jcell || n_cells <= 0) return cudaSuccess;
    std::vector<int32_t> vc((size_t)cell_off[n_cells]);
    for (int ci = 0; ci < n_cells; ++ci)
        for (int l = cell_off[ci]; l < cell_off[ci + 1]; ++l) vc[(size_t)l] = ci;
    cudaError_t e = cudaMemcpyAsync(c->ws + c->L.jcell, vc.data(), vc.size() * 4,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // vc is a host temporary
    return e;
}

extern "C" {

int lbib_workspace_size(const lbib_params* params, int32_t max_vertices, int32_t max_cells,
                        uint64_t* bytes_out) {
    std::string why;
    int rc = check_params(params, &why);
    if (rc) return fail(nullptr, rc, why);
    if (!bytes_out) return fail(nullptr, LBIB_E_PARAM, "bytes_out is NULL");
    Layout L;
    if (!make_layout(*params, max_vertices, max_cells, &L))
        return fail(nullptr, LBIB_E_PARAM, "invalid capacities");
    *bytes_out = L.total;
    return LBIB_OK;
}

int lbib_create(const lbib_params* params, int32_t max_vertices, int32_t max_cells,
                void* d_workspace, uint64_t bytes, void* cuda_stream, lbib_ctx** out) {
    std::string why;
    if (!out) return fail(nullptr, LBIB_E_PARAM, "out is NULL");
    *out = nullptr;
    int rc = check_params(params, &why);
    if (rc) return fail(nullptr, rc, why);
    Layout L;
    if (!make_layout(*params, max_vertices, max_cells, &L))
        return fail(nullptr, LBIB_E_PARAM, "invalid capacities");
    if (!d_workspace) return fail(nullptr, LBIB_E_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return fail(nullptr, LBIB_E_WORKSPACE, "workspace must be 256-byte aligned");
    if (bytes < L.total)
        return fail(nullptr, LBIB_E_WORKSPACE,
                    "workspace too small: need " + std::to_string(L.total) + " bytes");
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, d_workspace);
    if (e != cudaSuccess || (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(nullptr, LBIB_E_WORKSPACE, "workspace is not device memory");
    }
    lbib_ctx* c = new (std::nothrow) lbib_ctx();
    if (!c) return fail(nullptr, LBIB_E_PARAM, "out of host memory");
    c->p = *params;
    c->maxV = max_vertices;
    c->maxC = max_cells;
    c->ws = static_cast<char*>(d_workspace);
    c->bytes = bytes;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->L = L;
    fill_coefs(c->p, &c->kd);
    fill_coefs(c->p, &c->kf);
    c->l2_first = lattice_l2_first(c->p.precision, c->p.n_species, L.plane);
    e = launch_init_populations(c->p.precision, c->p.n_species, c->p.nx, c->p.ny, L.pitch,
                                L.plane, c->ws + L.f[0], c->ws + L.g[0], c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.force, 0, 2 * L.plane * L.cs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.u, 0, 2 * L.plane * L.cs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.id, 0xFF, L.plane * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.fmask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.lmask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.src, 0, align_up(L.plane, 8), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.smask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess && params->noflux_mask)
        e = cudaMemsetAsync(c->ws + L.dom, 0, L.plane * 4, c->stream);
    if (e == cudaSuccess && L.ncode)
        e = launch_make_ncode(c->at<int32_t>(L.dom), c->at<uint16_t>(L.ncode), params->nx,
                              params->ny, params->bc_y, L.pitch, c->stream);
    for (uint64_t off : {L.mrate, L.marea, L.msrc})
        if (e == cudaSuccess && off)
            e = cudaMemsetAsync(c->ws + off, 0, (size_t)8 * max_cells, c->stream);
    if (e == cudaSuccess && params->pressure_nodes)
        e = cudaMemsetAsync(c->ws + L.pnode, 0, align_up(L.plane, 8), c->stream);
    if (e == cudaSuccess && params->node_sources)
        e = cudaMemsetAsync(c->ws + L.nsrc, 0, L.plane * L.cs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.diag, 0, kDiagWords * 4, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && max_cells > 0)
        e = cudaHostAlloc(reinterpret_cast<void**>(&c->hstage), (size_t)max_cells * 9,
                          cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->hstage_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        lbib_destroy(c);
        return cuda_fail(nullptr, e, "lbib_create");
    }
    *out = c;
    return LBIB_OK;
}

int lbib_set_cells(lbib_ctx* c, int32_t n_cells, const int32_t* cell_off, const double* xy,
                   const double* rest_len, const double* k_spring, const double* pressure,
                   const uint8_t* src_flag) {
    NvtxRange nvtx_range("lbib_set_cells");
    if (!c) return LBIB_E_PARAM;
    {
        const cudaError_t fe = rb_fence(c, c->stream);
        if (fe != cudaSuccess) return cuda_fail(c, fe, "lbib_set_cells");
    }
    if (n_cells < 0 || n_cells > c->maxC) return fail(c, LBIB_E_CELLS, "n_cells exceeds capacity");
    if (n_cells > 0 && (!cell_off || !xy)) return fail(c, LBIB_E_CELLS, "cell_off and xy are required");
    int V = n_cells > 0 ? cell_off[n_cells] : 0;
    if (n_cells > 0 && cell_off[0] != 0) return fail(c, LBIB_E_CELLS, "cell_off[0] must be 0");
    for (int i = 0; i < n_cells; ++i) {
        int nv = cell_off[i + 1] - cell_off[i];
        if (nv < 3) return fail(c, LBIB_E_CELLS, "a cell needs at least 3 vertices");
        if (nv > kMaxVertsPerCell) return fail(c, LBIB_E_CELLS, "a cell has more than 1024 vertices");
    }
    if (V > c->maxV) return fail(c, LBIB_E_CELLS, "vertex count exceeds capacity");
    for (int i = 0; i < 2 * V; ++i)
        if (!std::isfinite(xy[i]) || std::fabs(xy[i]) > 1e9)
            return fail(c, LBIB_E_NONFINITE, "non-finite or out-of-range vertex position");
    for (int ci = 0; ci < n_cells; ++ci) {
        int a = cell_off[ci], b = cell_off[ci + 1];
        double xmn = xy[2 * a], xmx = xmn, ymn = xy[2 * a + 1], ymx = ymn, s = 0.0;
        for (int l = a; l < b; ++l) {
            int m = (l + 1 < b) ? l + 1 : a;
            xmn = std::fmin(xmn, xy[2 * l]); xmx = std::fmax(xmx, xy[2 * l]);
            ymn = std::fmin(ymn, xy[2 * l + 1]); ymx = std::fmax(ymx, xy[2 * l + 1]);
            s += (xy[2 * l] - xy[2 * a]) * (xy[2 * m + 1] - xy[2 * a + 1]) -
                 (xy[2 * m] - xy[2 * a]) * (xy[2 * l + 1] - xy[2 * a + 1]);
        }
        if (!(s > 0.0)) return fail(c, LBIB_E_CELLS, "cell polygons must be counter-clockwise");
        if (xmx - xmn > c->p.nx - 4 || ymx - ymn > c->p.ny - 4)
            return fail(c, LBIB_E_CELLS, "a cell is larger than the lattice");
    }
    std::vector<double> L0((size_t)V), kk((size_t)V, 0.0), pp((size_t)n_cells, 0.0);
    std::vector<uint8_t> sf((size_t)n_cells, 0);
    for (int ci = 0; ci < n_cells; ++ci) {
        int a = cell_off[ci], b = cell_off[ci + 1];
        for (int l = a; l < b; ++l) {
            int m = (l + 1 < b) ? l + 1 : a;
            double dx = xy[2 * m] - xy[2 * l], dy = xy[2 * m + 1] - xy[2 * l + 1];
            L0[l] = rest_len ? rest_len[l] : std::sqrt(dx * dx + dy * dy);
            if (k_spring) kk[l] = k_spring[l];
        }
        if (pressure) pp[ci] = pressure[ci];
        if (src_flag) sf[ci] = src_flag[ci];
    }
    const Layout& L = c->L;
    cudaError_t e = cudaSuccess;
    if (V > 0) {
        e = cudaMemcpyAsync(c->ws + L.xy, xy, (size_t)V * 16, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + L.L0, L0.data(), (size_t)V * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + L.k, kk.data(), (size_t)V * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + L.off, cell_off, (size_t)(n_cells + 1) * 4,
                                cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + L.pres, pp.data(), (size_t)n_cells * 8, cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + L.srcf, sf.data(), (size_t)n_cells, cudaMemcpyHostToDevice,
                                c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = upload_vertex_cells(c, n_cells, cell_off);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_cells");
    c->nstep = 0;
    c->nV = V;
    c->nC = n_cells;
    c->maxv_cell = 0;
    for (int ci = 0; ci < n_cells; ++ci)
        c->maxv_cell = std::max(c->maxv_cell, cell_off[ci + 1] - cell_off[ci]);
    c->vforce_valid = false;
    drop_graphs(c);
    return LBIB_OK;
}

int lbib_set_domains(lbib_ctx* c, const int32_t* labels) {
    if (!c) return LBIB_E_PARAM;
    if (!c->p.noflux_mask) return fail(c, LBIB_E_STATE, "the context has no confined species");
    const Layout& L = c->L;
    cudaError_t e;
    if (labels)
        e = cudaMemcpy2DAsync(c->ws + L.dom, (size_t)L.pitch * 4, labels, (size_t)c->p.nx * 4,
                              (size_t)c->p.nx * 4, (size_t)c->p.ny, cudaMemcpyHostToDevice,
                              c->stream);
    else
        e = cudaMemsetAsync(c->ws + L.dom, 0, L.plane * 4, c->stream);
    if (e == cudaSuccess && L.ncode)
        e = launch_make_ncode(c->at<int32_t>(L.dom), c->at<uint16_t>(L.ncode), c->p.nx, c->p.ny,
                              c->p.bc_y, L.pitch, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_domains");
    // the moments were kept where the old closures read them
    c->mom_valid = false;
    return LBIB_OK;
}

int lbib_set_mass_sources(lbib_ctx* c, const double* rate, const double* target_area) {
    if (!c) return LBIB_E_PARAM;
    if (!c->p.mass_sources || !c->L.mrate)
        return fail(c, LBIB_E_STATE, "the context has no mass sources");
    const Layout& L = c->L;
    const size_t nc = (size_t)c->nC;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && nc > 0) {
        if (rate)
            e = cudaMemcpyAsync(c->ws + L.mrate, rate, nc * 8, cudaMemcpyHostToDevice, c->stream);
        else
            e = cudaMemsetAsync(c->ws + L.mrate, 0, nc * 8, c->stream);
    }
    if (e == cudaSuccess && nc > 0 && target_area)
        e = cudaMemcpyAsync(c->ws + L.marea, target_area, nc * 8, cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_mass_sources");
    if (c->mass_ctrl != (target_area != nullptr)) {
        drop_graphs(c);  // the captured steps hold the other controller setting
        c->mass_ctrl = target_area != nullptr;
    }
    return LBIB_OK;
}

int lbib_set_pressure_nodes(lbib_ctx* c, const uint8_t* mask) {
    if (!c) return LBIB_E_PARAM;
    if (!c->p.pressure_nodes) return fail(c, LBIB_E_STATE, "the context has no pressure nodes");
    const Layout& L = c->L;
    cudaError_t e;
    if (mask)
        e = cudaMemcpy2DAsync(c->ws + L.pnode, (size_t)L.pitch, mask, (size_t)c->p.nx,
                              (size_t)c->p.nx, (size_t)c->p.ny, cudaMemcpyHostToDevice,
                              c->stream);
    else
        e = cudaMemsetAsync(c->ws + L.pnode, 0, L.plane, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_pressure_nodes");
    return LBIB_OK;
}

int lbib_set_node_sources(lbib_ctx* c, const double* S) {
    if (!c) return LBIB_E_PARAM;
    if (!c->p.node_sources) return fail(c, LBIB_E_STATE, "the context has no node sources");
    const Layout& L = c->L;
    const size_t nx = (size_t)c->p.nx, ny = (size_t)c->p.ny;
    cudaError_t e = cudaSuccess;
    if (!S) {
        e = cudaMemsetAsync(c->ws + L.nsrc, 0, L.plane * L.cs, c->stream);
    } else if (L.cs == 8) {
        e = cudaMemcpy2DAsync(c->ws + L.nsrc, (size_t)L.pitch * 8, S, nx * 8, nx * 8, ny,
                              cudaMemcpyHostToDevice, c->stream);
    } else {
        // FP32 / FP16 storage compute in FP32: convert on the host
        std::vector<float> f(nx * ny);
        for (size_t t = 0; t < f.size(); ++t) f[t] = (float)S[t];
        e = cudaMemcpy2DAsync(c->ws + L.nsrc, (size_t)L.pitch * 4, f.data(), nx * 4, nx * 4, ny,
                              cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // f is a host temporary
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_node_sources");
    return LBIB_OK;
}

int lbib_set_lattice_variant(lbib_ctx* c, int32_t nodes_per_thread) {
    if (!c) return LBIB_E_PARAM;
    if (nodes_per_thread != 0 && nodes_per_thread != 1 && nodes_per_thread != 2 &&
        nodes_per_thread != 4)
        return fail(c, LBIB_E_PARAM, "nodes_per_thread must be 0, 1, 2 or 4");
    if (nodes_per_thread != c->lattice_npt) {
        // the captured step graphs hold the other kernel
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_lattice_variant");
        drop_graphs(c);
        c->lattice_npt = nodes_per_thread;
    }
    return LBIB_OK;
}

int lbib_set_cell_params(lbib_ctx* c, const double* pressure, const uint8_t* src_flag) {
    if (!c) return LBIB_E_PARAM;
    if (c->nC == 0 || (!pressure && !src_flag)) return LBIB_OK;
    // the host arrays are copied into the context's pinned staging buffer
    // (free again once the previous upload has run) and uploaded
    // asynchronously on the context stream: the caller may reuse them at once
    cudaError_t e = cudaSuccess;
    if (c->hstage_pending) e = cudaEventSynchronize(c->hstage_done);
    const size_t nc = (size_t)c->nC;
    if (e == cudaSuccess && pressure) {
        std::memcpy(c->hstage, pressure, nc * 8);
        e = cudaMemcpyAsync(c->ws + c->L.pres, c->hstage, nc * 8, cudaMemcpyHostToDevice,
                            c->stream);
    }
    if (e == cudaSuccess && src_flag) {
        std::memcpy(c->hstage + nc * 8, src_flag, nc);
        e = cudaMemcpyAsync(c->ws + c->L.srcf, c->hstage + nc * 8, nc, cudaMemcpyHostToDevice,
                            c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->hstage_done, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_cell_params");
    c->hstage_pending = true;
    return LBIB_OK;
}

int lbib_set_species(lbib_ctx* c, int32_t s, const double* phi) {
    if (!c) return LBIB_E_PARAM;
    if (s < 0 || s >= c->p.n_species) return fail(c, LBIB_E_PARAM, "species index out of range");
    if (!phi) return fail(c, LBIB_E_PARAM, "phi is NULL");
    const size_t N = (size_t)c->p.nx * c->p.ny;
    // The host field is staged in the force_out planes (2 planes of the compute
    // type hold at least nx*ny doubles); they only carry the last step's output.
    double* stage = c->at<double>(c->L.force_out);
    if ((uint64_t)N * 8 > (uint64_t)2 * c->L.plane * c->L.cs)
        return fail(c, LBIB_E_STATE, "staging area too small");
    cudaError_t e = cudaMemcpyAsync(stage, phi, N * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_set_species(c->p.precision, c->p.n_species, s, c->p.nx, c->p.ny, c->L.pitch,
                               c->L.plane, stage, c->ws + c->L.g[c->cur], coefs_of(c), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_species");
    c->fields_valid = false;
    c->mom_valid = false;
    return LBIB_OK;
}

int lbib_step(lbib_ctx* c, int32_t n_steps) {
    NvtxRange nvtx_range("lbib_step");
    if (!c) return LBIB_E_PARAM;
    if (n_steps < 0) return fail(c, LBIB_E_PARAM, "n_steps must be >= 0");
    if (n_steps == 0) return LBIB_OK;
    {
        const cudaError_t fe = rb_fence(c, c->stream);
        if (fe != cudaSuccess) return cuda_fail(c, fe, "lbib_step");
    }
    cudaError_t e = ensure_moments(c);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_step");
    const bool ib = c->nC > 0;
    if (ib && c->p.junction_period > 0) {
        e = run_with_junctions(c, n_steps, true, [](int, auto&& fn) { return fn(); });
        if (e != cudaSuccess) return cuda_fail(c, e, "lbib_step");
        c->fields_valid = true;
        c->vforce_valid = true;
        return LBIB_OK;
    }
    // prep of the first step (labels, forces, spreading from X^n)
    if (ib) e = enqueue_ib(c, false, true, n_steps == 1);
    int left = n_steps;
    // full two-step chunks through the graph, keeping the last two steps apart
    // (they write the vertex forces and the output fields)
    bool graphed = false;
    while (e == cudaSuccess && left > 3) {
        cudaGraphExec_t g;
        e = get_chunk_graph(c, c->cur, &g);
        if (e == cudaSuccess) e = cudaGraphLaunch(g, c->stream);
        graphed = true;
        left -= 2;
    }
    // the remaining steps as single launches: a launch that directly follows
    // the other kernel of the step (not a graph) is programmatic
    bool follows_kernel = ib && !graphed;
    while (e == cudaSuccess && left > 0) {
        const bool last = (left == 1);
        e = enqueue_lattice(c, c->cur, last, follows_kernel);
        if (e == cudaSuccess && ib) e = enqueue_ib(c, true, !last, left == 2, true);
        follows_kernel = ib;
        c->cur = 1 - c->cur;
        --left;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_step");
    c->fields_valid = true;
    c->vforce_valid = ib;
    return LBIB_OK;
}

int lbib_advance(lbib_ctx* c, int32_t n_steps) {
    NvtxRange nvtx_range("lbib_advance");
    if (!c) return LBIB_E_PARAM;
    if (n_steps < 0) return fail(c, LBIB_E_PARAM, "n_steps must be >= 0");
    if (n_steps == 0) return LBIB_OK;
    const bool ib = c->nC > 0;
    // steps with junctions are launched one by one anyway
    if (ib && c->p.junction_period > 0) return lbib_step(c, n_steps);
    cudaError_t e = ensure_moments(c);
    if (ib && e == cudaSuccess) e = enqueue_ib(c, false, true, false);
    int left = n_steps;
    // an odd count starts with one directly launched step (programmatic after
    // the prep); its IB launch moves, and preps unless it is the only step
    // a pending readback of the vertex positions and areas runs beside the
    // prep and the lattice update; the first move waits for it
    if (left % 2 == 1) {
        if (e == cudaSuccess) e = enqueue_lattice(c, c->cur, false, ib);
        if (e == cudaSuccess && ib) {
            const bool fenced = c->rb_pending;
            e = rb_fence(c, c->stream);
            // after an event wait the move is not a programmatic launch
            if (e == cudaSuccess) e = enqueue_ib(c, true, left > 1, false, !fenced);
        }
        c->cur = 1 - c->cur;
        --left;
    }
    if (e == cudaSuccess && left > 0) e = rb_fence(c, c->stream);
    while (e == cudaSuccess && left > 0) {
        cudaGraphExec_t g;
        e = get_chunk_graph(c, c->cur, &g, left == 2);
        if (e == cudaSuccess) e = cudaGraphLaunch(g, c->stream);
        left -= 2;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_advance");
    // the lattice fields, labels and vertex forces of the last step were not written
    c->fields_valid = false;
    c->vforce_valid = false;
    return LBIB_OK;
}

int lbib_step_profiled(lbib_ctx* c, int32_t n_steps, double* ms_out) {
    if (!c || !ms_out) return LBIB_E_PARAM;
    if (n_steps <= 0) return fail(c, LBIB_E_PARAM, "n_steps must be > 0");
    {
        const cudaError_t fe = rb_fence(c, c->stream);
        if (fe != cudaSuccess) return cuda_fail(c, fe, "lbib_step_profiled");
    }
    const bool ib = c->nC > 0;
    const bool junctions = ib && c->p.junction_period > 0;
    // one event before and after every launch: 2 per launch (with junctions
    // at most a renewal, a prep, a lattice update and a move per step)
    const int n_launch = junctions ? 4 * n_steps + 2 : n_steps + (ib ? n_steps + 1 : 0);
    std::vector<cudaEvent_t> ev((size_t)2 * n_launch, nullptr);
    std::vector<int> kind((size_t)n_launch, 0);
    cudaError_t e = ensure_moments(c);
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    int li = 0;
    auto timed = [&](int k, auto&& fn) {
        if (e != cudaSuccess) return;
        e = cudaEventRecord(ev[2 * li], c->stream);
        if (e == cudaSuccess) e = fn();
        if (e == cudaSuccess) e = cudaEventRecord(ev[2 * li + 1], c->stream);
        kind[li++] = k;
    };
    if (junctions) {
        run_with_junctions(c, n_steps, false, [&](int k, auto&& fn) {
            timed(k, fn);
            return e;
        });
    } else {
        if (ib) timed(1, [&] { return enqueue_ib(c, false, true, n_steps == 1); });
        for (int left = n_steps; left > 0 && e == cudaSuccess; --left) {
            const bool last = (left == 1);
            timed(0, [&] { return enqueue_lattice(c, c->cur, last); });
            if (ib) timed(1, [&] { return enqueue_ib(c, true, !last, left == 2); });
            c->cur = 1 - c->cur;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    ms_out[0] = ms_out[1] = 0.0;
    for (int i = 0; i < li && e == cudaSuccess; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
        ms_out[kind[i]] += ms;
    }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_step_profiled");
    c->fields_valid = true;
    c->vforce_valid = ib;
    return LBIB_OK;
}

// the status the device-side diagnostic words report (checking build,
// non-finite fields, blown-up cells)
static int diag_status(lbib_ctx* c, const uint32_t* diag) {
    if (diag[kDiagCheck]) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "checking build: an access failed its bounds or alignment check "
                      "(site %u, address low bits 0x%08x) and was skipped",
                      diag[kDiagCheckSite], diag[kDiagCheckAddr]);
        return fail(c, LBIB_E_CHECK, msg);
    }
    if (diag[kDiagNonFinite])
        return fail(c, LBIB_E_NONFINITE, "a non-finite density or velocity was produced");
    if (diag[kDiagGeometry])
        return fail(c, LBIB_E_NONFINITE, "a cell became non-finite or larger than the lattice");
    return LBIB_OK;
}

int lbib_get_fields(lbib_ctx* c, uint32_t which, double* rho, double* ux, double* uy, double* phi,
                    double* xy, double* area, int32_t* id, double* force, double* vforce) {
    NvtxRange nvtx_range("lbib_get_fields");
    if (!c) return LBIB_E_PARAM;
    {
        const cudaError_t fe = rb_fence(c, c->stream);
        if (fe != cudaSuccess) return cuda_fail(c, fe, "lbib_get_fields");
    }
    const uint32_t lattice_bits = LBIB_RHO | LBIB_U | LBIB_PHI | LBIB_ID | LBIB_FORCE;
    if ((which & lattice_bits) && !c->fields_valid)
        return fail(c, LBIB_E_STATE, "no completed step since the last create or reset");
    if ((which & (LBIB_ID | LBIB_FORCE)) && c->nC == 0)
        return fail(c, LBIB_E_STATE, "labels and spread force need cells");
    if ((which & LBIB_VFORCE) && c->nV > 0 && !c->vforce_valid)
        return fail(c, LBIB_E_STATE, "no vertex forces computed yet");
    const Layout& L = c->L;
    const int nx = c->p.nx, ny = c->p.ny, S = c->p.n_species;
    const size_t N = (size_t)nx * ny;
    cudaError_t e = cudaSuccess;
    // Every copy is enqueued first and the stream synchronised once.  Lattice
    // planes are copied raw (storage pitch, compute type) to host memory and
    // converted there, so no device scratch is needed; vertex data and areas
    // go straight to the caller's buffers.
    std::vector<char> r_rho, r_u, r_phi, r_id, r_force;
    auto fetch = [&](std::vector<char>& raw, uint64_t off, size_t bytes) {
        raw.resize(bytes);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(raw.data(), c->ws + off, bytes, cudaMemcpyDeviceToHost, c->stream);
    };
    if (which & LBIB_RHO) fetch(r_rho, L.rho, (size_t)L.plane * L.cs);
    if (which & LBIB_U) fetch(r_u, L.u, (size_t)2 * L.plane * L.cs);
    if ((which & LBIB_PHI) && S > 0) fetch(r_phi, L.phi, (size_t)S * L.plane * L.cs);
    if (which & LBIB_ID) fetch(r_id, L.id_out, (size_t)L.plane * 4);
    if (which & LBIB_FORCE) fetch(r_force, L.force_out, (size_t)2 * L.plane * L.cs);
    if ((which & LBIB_X) && c->nV > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(xy, c->ws + L.xy, (size_t)c->nV * 16, cudaMemcpyDeviceToHost, c->stream);
    if ((which & LBIB_VFORCE) && c->nV > 0 && e == cudaSuccess)
        e = cudaMemcpyAsync(vforce, c->ws + L.vforce, (size_t)c->nV * 16, cudaMemcpyDeviceToHost,
                            c->stream);
    if ((which & LBIB_AREA) && c->nC > 0 && e == cudaSuccess) {
        e = launch_areas(c->at<double2>(L.xy), c->at<int32_t>(L.off), c->nC, c->at<double>(L.area),
                         c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(area, c->ws + L.area, (size_t)c->nC * 8, cudaMemcpyDeviceToHost,
                                c->stream);
    }
    // the device-side diagnostics
    uint32_t diag[kDiagCheckAddr + 1] = {0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(diag, c->ws + L.diag, sizeof(diag), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_get_fields");

    auto val = [&](const std::vector<char>& raw, int64_t idx) -> double {
        return c->L.cs == 8 ? reinterpret_cast<const double*>(raw.data())[idx]
                            : (double)reinterpret_cast<const float*>(raw.data())[idx];
    };
    if (which & LBIB_RHO)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) rho[(size_t)y * nx + x] = val(r_rho, (int64_t)y * L.pitch + x);
    if (which & LBIB_U)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t n = (int64_t)y * L.pitch + x;
                if (ux) ux[(size_t)y * nx + x] = val(r_u, 2 * n);
                if (uy) uy[(size_t)y * nx + x] = val(r_u, 2 * n + 1);
            }
    if ((which & LBIB_PHI) && S > 0)
        for (int s = 0; s < S; ++s)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x)
                    phi[(size_t)s * N + (size_t)y * nx + x] =
                        val(r_phi, (int64_t)s * L.plane + (int64_t)y * L.pitch + x);
    if (which & LBIB_ID) {
        const uint32_t* v = reinterpret_cast<const uint32_t*>(r_id.data());
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint32_t t = v[(int64_t)y * L.pitch + x];
                id[(size_t)y * nx + x] = (t == kOutside) ? 0 : (int32_t)(t >> 4) + 1;
            }
    }
    if (which & LBIB_FORCE)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t n = (int64_t)y * L.pitch + x;
                force[2 * ((size_t)y * nx + x)] = val(r_force, 2 * n);
                force[2 * ((size_t)y * nx + x) + 1] = val(r_force, 2 * n + 1);
            }
    return diag_status(c, diag);
}

// Asynchronous readback of the cell outputs.  The copies run on the
// context's copy stream after an event of the context stream, so that the
// steps enqueued afterwards overlap them; every call that writes the vertex
// positions or the areas orders itself after rb_done (rb_fence).
int lbib_get_cells_async(lbib_ctx* c, uint32_t which, double* xy, double* area) {
    NvtxRange nvtx_range("lbib_get_cells_async");
    if (!c) return LBIB_E_PARAM;
    if (which & ~(LBIB_X | LBIB_AREA))
        return fail(c, LBIB_E_PARAM, "lbib_get_cells_async: only LBIB_X and LBIB_AREA");
    if (((which & LBIB_X) && c->nV > 0 && !xy) || ((which & LBIB_AREA) && c->nC > 0 && !area))
        return fail(c, LBIB_E_PARAM, "lbib_get_cells_async: NULL output buffer");
    // one readback at a time: the previous one ends first (its status stands)
    if (c->rb_pending) {
        const int rc = lbib_wait_readback(c);
        if (rc != LBIB_OK) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (!c->rb_stream) {
        e = cudaStreamCreateWithFlags(&c->rb_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->rb_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->rb_done, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void**>(&c->rb_diag), (kDiagCheckAddr + 1) * 4,
                              cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(c, e, "lbib_get_cells_async");
    }
    const Layout& L = c->L;
    if ((which & LBIB_AREA) && c->nC > 0)
        e = launch_areas(c->at<double2>(L.xy), c->at<int32_t>(L.off), c->nC, c->at<double>(L.area),
                         c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->rb_ready, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->rb_stream, c->rb_ready, 0);
    if (e == cudaSuccess && (which & LBIB_X) && c->nV > 0)
        e = cudaMemcpyAsync(xy, c->ws + L.xy, (size_t)c->nV * 16, cudaMemcpyDeviceToHost,
                            c->rb_stream);
    if (e == cudaSuccess && (which & LBIB_AREA) && c->nC > 0)
        e = cudaMemcpyAsync(area, c->ws + L.area, (size_t)c->nC * 8, cudaMemcpyDeviceToHost,
                            c->rb_stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->rb_diag, c->ws + L.diag, (kDiagCheckAddr + 1) * 4,
                            cudaMemcpyDeviceToHost, c->rb_stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->rb_done, c->rb_stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_get_cells_async");
    c->rb_pending = true;
    return LBIB_OK;
}

int lbib_wait_readback(lbib_ctx* c) {
    NvtxRange nvtx_range("lbib_wait_readback");
    if (!c) return LBIB_E_PARAM;
    if (!c->rb_pending) return LBIB_OK;
    const cudaError_t e = cudaEventSynchronize(c->rb_done);
    c->rb_pending = false;
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_wait_readback");
    return diag_status(c, c->rb_diag);
}

int lbib_get_sizes(const lbib_ctx* c, int32_t* n_vertices, int32_t* n_cells) {
    if (!c) return LBIB_E_PARAM;
    if (n_vertices) *n_vertices = c->nV;
    if (n_cells) *n_cells = c->nC;
    return LBIB_OK;
}

// state: populations of the current buffer (f then g), then xy, L0, k, off,
// pres, srcf, then a small header {cur-independent}.
// the no-flux closure's moments of the previous step (part of the state)
static uint64_t mom_bytes(const lbib_ctx* c) {
    return c->L.ncode ? (uint64_t)3 * c->p.n_species * c->L.plane * c->L.cs : 0;
}

static uint64_t state_bytes(const lbib_ctx* c) {
    const Layout& L = c->L;
    uint64_t P = (uint64_t)L.plane * L.es;
    return 16 + 9 * P + (uint64_t)5 * c->p.n_species * P + (uint64_t)c->maxV * 32 +
           (uint64_t)(c->maxC + 1) * 4 + (uint64_t)c->maxC * 9 + mom_bytes(c);
}

int lbib_state_size(const lbib_ctx* c, uint64_t* bytes_out) {
    if (!c || !bytes_out) return LBIB_E_PARAM;
    *bytes_out = state_bytes(c);
    return LBIB_OK;
}

int lbib_get_state(lbib_ctx* c, void* host, uint64_t bytes) {
    if (!c || !host) return LBIB_E_PARAM;
    if (bytes < state_bytes(c)) return fail(c, LBIB_E_PARAM, "state buffer too small");
    const Layout& L = c->L;
    char* h = static_cast<char*>(host);
    {
        cudaError_t em = ensure_moments(c);
        if (em != cudaSuccess) return cuda_fail(c, em, "lbib_get_state");
    }
    int32_t hdr[4] = {c->nV, c->nC, c->p.precision, c->p.n_species};
    std::memcpy(h, hdr, 16);
    uint64_t o = 16, P = (uint64_t)L.plane * L.es;
    struct Piece { uint64_t off, bytes; } pieces[] = {
        {L.f[c->cur], 9 * P}, {L.g[c->cur], (uint64_t)5 * c->p.n_species * P},
        {L.xy, (uint64_t)c->maxV * 16}, {L.L0, (uint64_t)c->maxV * 8}, {L.k, (uint64_t)c->maxV * 8},
        {L.off, (uint64_t)(c->maxC + 1) * 4}, {L.pres, (uint64_t)c->maxC * 8},
        {L.srcf, (uint64_t)c->maxC}, {L.mom[c->cur], mom_bytes(c)}};
    cudaError_t e = cudaSuccess;
    for (auto& pc : pieces) {
        if (pc.bytes && e == cudaSuccess)
            e = cudaMemcpyAsync(h + o, c->ws + pc.off, pc.bytes, cudaMemcpyDeviceToHost, c->stream);
        o += pc.bytes;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_get_state");
    return LBIB_OK;
}

int lbib_set_state(lbib_ctx* c, const void* host, uint64_t bytes) {
    if (!c || !host) return LBIB_E_PARAM;
    {
        const cudaError_t fe = rb_fence(c, c->stream);
        if (fe != cudaSuccess) return cuda_fail(c, fe, "lbib_set_state");
    }
    if (bytes < state_bytes(c)) return fail(c, LBIB_E_PARAM, "state buffer too small");
    const char* h = static_cast<const char*>(host);
    int32_t hdr[4];
    std::memcpy(hdr, h, 16);
    if (hdr[0] < 0 || hdr[0] > c->maxV || hdr[1] < 0 || hdr[1] > c->maxC ||
        hdr[2] != c->p.precision || hdr[3] != c->p.n_species)
        return fail(c, LBIB_E_STATE, "state does not match this context");
    const Layout& L = c->L;
    uint64_t o = 16, P = (uint64_t)L.plane * L.es;
    c->cur = 0;
    struct Piece { uint64_t off, bytes; } pieces[] = {
        {L.f[0], 9 * P}, {L.g[0], (uint64_t)5 * c->p.n_species * P},
        {L.xy, (uint64_t)c->maxV * 16}, {L.L0, (uint64_t)c->maxV * 8}, {L.k, (uint64_t)c->maxV * 8},
        {L.off, (uint64_t)(c->maxC + 1) * 4}, {L.pres, (uint64_t)c->maxC * 8},
        {L.srcf, (uint64_t)c->maxC}, {L.mom[0], mom_bytes(c)}};
    cudaError_t e = cudaSuccess;
    for (auto& pc : pieces) {
        if (pc.bytes && e == cudaSuccess)
            e = cudaMemcpyAsync(c->ws + pc.off, h + o, pc.bytes, cudaMemcpyHostToDevice, c->stream);
        o += pc.bytes;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.force, 0, 2 * L.plane * L.cs, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.id, 0xFF, L.plane * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.fmask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.lmask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.src, 0, align_up(L.plane, 8), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ws + L.smask, 0, mask_words(L.plane) * 4, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbib_set_state");
    c->nV = hdr[0];
    c->nC = hdr[1];
    {   // the largest cell, from the cell offsets of the state
        const int32_t* off = reinterpret_cast<const int32_t*>(
            h + 16 + 9 * P + (uint64_t)5 * c->p.n_species * P + (uint64_t)c->maxV * 32);
        c->maxv_cell = 0;
        for (int ci = 0; ci < c->nC; ++ci) c->maxv_cell = std::max(c->maxv_cell, off[ci + 1] - off[ci]);
        cudaError_t ev = upload_vertex_cells(c, c->nC, off);
        if (ev != cudaSuccess) return cuda_fail(c, ev, "lbib_set_state");
    }
    c->nstep = 0;
    c->fields_valid = false;
    c->vforce_valid = false;
    c->mom_valid = true;  // restored with the populations
    drop_graphs(c);
    return LBIB_OK;
}

void lbib_destroy(lbib_ctx* c) {
    if (!c) return;
    if (c->rb_done) cudaEventSynchronize(c->rb_done);  // a pending readback's copies
    if (c->rb_stream) cudaStreamDestroy(c->rb_stream);
    if (c->rb_ready) cudaEventDestroy(c->rb_ready);
    if (c->rb_done) cudaEventDestroy(c->rb_done);
    if (c->rb_diag) cudaFreeHost(c->rb_diag);
    drop_graphs(c);
    if (c->hstage_done) {
        cudaEventSynchronize(c->hstage_done);
        cudaEventDestroy(c->hstage_done);
    }
    if (c->hstage) cudaFreeHost(c->hstage);
    delete c;
}

const char* lbib_last_error(const lbib_ctx* c) {
    return c ? c->err.c_str() : g_create_err.c_str();
}

const char* lbib_status_string(int status) {
    switch (status) {
        case LBIB_OK: return "LBIB_OK";
        case LBIB_E_PARAM: return "LBIB_E_PARAM";
        case LBIB_E_WORKSPACE: return "LBIB_E_WORKSPACE";
        case LBIB_E_CELLS: return "LBIB_E_CELLS";
        case LBIB_E_NONFINITE: return "LBIB_E_NONFINITE";
        case LBIB_E_TIMEOUT: return "LBIB_E_TIMEOUT";
        case LBIB_E_CUDA: return "LBIB_E_CUDA";
        case LBIB_E_STATE: return "LBIB_E_STATE";
        case LBIB_E_CHECK: return "LBIB_E_CHECK";
        default: return "LBIB_E_UNKNOWN";
    }
}

}  // extern "C"
