// ensemble.cu -- a batch of independent tissues advanced together by one
// persistent, cooperative kernel launch per lbib_ensemble_step() call.
//
// Every tissue is an ordinary context (its own slice of the ensemble's
// workspace, its own parameters: lattice size, tau, boundary, springs), so
// the per-tissue calls (lbib_set_cells, lbib_get_fields, state) work on it.
// lbib_ensemble_step(n) runs, for all tissues at once, the same sequence as
// lbib_step(n): the IB prep, then per step the lattice update of every node
// of every tissue and the IB move/prep of every cell, separated by grid-wide
// barriers.  Work is dealt out in items -- lattice items of `nodes_per_item`
// nodes (rows padded to 32 so a warp stays in one row) and one item per cell
// -- strided over the persistent CTAs, which balances tissues of very
// different sizes.  The launch is captured once per step count into a CUDA
// graph and replayed.
//
// The split schedule runs the same items as two kernels per step instead --
// one lattice launch over every lattice item of every tissue (128-thread
// CTAs held to the standalone lattice kernel's registers, so an SM keeps
// twice the warps, and loads, of the persistent kernel in flight) and one IB
// launch over every cell -- ordered by programmatic dependent launches in
// place of the grid barriers: each kernel issues its loads of what the launch
// two back wrote before it waits on the launch just before, as the
// single-tissue steps do.  All 2n + 1 launches of n steps are one graph.
// The schedule and the two launch parameters (nodes per item, and CTAs per SM
// of the persistent kernel) are chosen by lbib_ensemble_tune(), which times
// the candidates.
//
// The grid barrier spins on a generation word with a bounded wait (a
// globaltimer limit of about one second): if a barrier cannot complete, the
// CTA records the error and every CTA leaves at its next barrier, so the
// launch always ends; lbib_ensemble_status() reports LBIB_E_TIMEOUT.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "ib_cell.cuh"
#include "lattice_kernel.cuh"
#include "lbib_ctx.cuh"

namespace lbib {

struct TissueDev {
    LatticeArgs la;    // parity-0 buffers: fsrc = f[0], fdst = f[1] (swapped per step)
    IBArgs ia;
    Coefs<float> k;
    int bc_y;
    int nxr;           // row length padded to a multiple of 32
    int cur;           // buffer parity at the start of the launch
    int pad;
};

static_assert(sizeof(TissueDev) % 4 == 0 && sizeof(IBArgs) % 4 == 0,
              "the tables are copied to shared memory in 4-byte words");

struct EnsArgs {
    const TissueDev* tis;
    const int* item_pfx;  // n + 1 prefix sums of lattice items
    const int* cell_pfx;  // n + 1 prefix sums of cells
    int n, n_steps, nodes_per_item, total_items, total_cells;
    int maxv;             // vertex arrays of each cell slot in shared memory
    int cell_threads;     // threads per cell in the IB phase (64 or 128)
    unsigned* bar;        // [0] arrival count, [1] generation, [2] error flag
    unsigned nblocks;     // CTAs the barrier waits for
};

constexpr unsigned long long kBarrierLimitNs = 1000000000ull;  // one second

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait.  Returns false (for every thread of
// the CTA) when the ensemble's error flag is set.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        volatile unsigned* verr = bar + 2;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g) {
                if (*verr) break;
                if (global_ns() - t0 > kBarrierLimitNs) {
                    atomicOr(bar + 2, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        // one reading of the error flag for the whole CTA, so that its threads
        // leave together
        s_ok = *(volatile unsigned*)(bar + 2) == 0u ? 1u : 0u;
    }
    __syncthreads();
    return s_ok != 0u;
}

__device__ __forceinline__ int find_tissue(const int* pfx, int n, int item) {
    int lo = 0, hi = n;  // pfx[lo] <= item < pfx[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pfx[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The IB phase runs several cells at a time per CTA: two per CTA (128-thread
// halves), or four (64-thread quarters) when no cell has more than 64
// vertices, each group with its own named barrier and its own slot of dynamic
// shared memory (fixed part + maxv vertices).  The per-cell work is a chain of
// dependent steps, so more cells in flight per SM shorten the phase.
__host__ __device__ inline int ens_cell_threads(int maxv) { return maxv <= 64 ? 64 : 128; }

__host__ __device__ inline size_t ens_cell_smem(int maxv) {
    return (size_t)kIBSmemFixed + (size_t)maxv * kIBSmemPerVertex;
}

template <int S, int FORCING>
__global__ void __launch_bounds__(kIBThreads, 3) ensemble_kernel(EnsArgs e) {
    extern __shared__ __align__(16) unsigned char ens_smem[];
    __shared__ TissueDev td;
    __shared__ int s_t;
    const int tid = threadIdx.x;
    const int cgroups = kIBThreads / e.cell_threads;
    const int half = tid / e.cell_threads, htid = tid % e.cell_threads;
    const IBShared32 view =
        ib_shared32_view(ens_smem + (size_t)half * ens_cell_smem(e.maxv), e.maxv);
    if (tid == 0) s_t = -1;

    auto load_tissue = [&](int t) {
        __syncthreads();
        if (t != s_t) {
            const int* src = reinterpret_cast<const int*>(e.tis + t);
            int* dst = reinterpret_cast<int*>(&td);
            for (int i = tid; i < (int)(sizeof(TissueDev) / 4); i += blockDim.x) dst[i] = src[i];
            __syncthreads();
            if (tid == 0) s_t = t;
        }
        __syncthreads();
    };

    auto ib_phase = [&](int move, int prep, int vforce) {
        for (int item = blockIdx.x * cgroups + half; item < e.total_cells;
             item += gridDim.x * cgroups) {
            const int t = find_tissue(e.cell_pfx, e.n, item);
            IBArgs a = e.tis[t].ia;
            a.do_move = move;
            a.do_prep = prep;
            a.write_vforce = vforce;
            a.do_ids = vforce;  // the prep of the output step writes the labels too
            if (e.cell_threads == 64)
                ib_cell_f32<64, false, false, false>(a, item - e.cell_pfx[t], view, htid,
                                                     1 + half);
            else
                ib_cell_f32<128, false, false, false>(a, item - e.cell_pfx[t], view, htid,
                                                      1 + half);
        }
    };

    auto lattice_phase = [&](int step, int out) {
        for (int item = blockIdx.x; item < e.total_items; item += gridDim.x) {
            const int t = find_tissue(e.item_pfx, e.n, item);
            load_tissue(t);
            LatticeArgs a = td.la;
            const int p = (td.cur + step) & 1;
            if (p) {
                a.fsrc = td.la.fdst;
                a.fdst = const_cast<void*>(td.la.fsrc);
                a.gsrc = td.la.gdst;
                a.gdst = const_cast<void*>(td.la.gsrc);
            }
            a.out = out;
            const int64_t v0 = (int64_t)(item - e.item_pfx[t]) * e.nodes_per_item;
            for (int v = tid; v < e.nodes_per_item; v += blockDim.x) {
                const int64_t vv = v0 + v;
                const int y = (int)(vv / td.nxr), x = (int)(vv - (int64_t)y * td.nxr);
                if (y >= a.ny || x >= a.nx) continue;
                if (td.bc_y)
                    lattice_node<float, float, S, true, FORCING, false>(a, td.k, x, y);
                else
                    lattice_node<float, float, S, false, FORCING, false>(a, td.k, x, y);
            }
        }
    };

    // the sequence of lbib_step(n): prep, then per step lattice + move/prep
    ib_phase(0, 1, e.n_steps == 1);
    if (!grid_barrier(e.bar, e.nblocks)) return;
    for (int s = 0; s < e.n_steps; ++s) {
        const bool last = (s == e.n_steps - 1);
        lattice_phase(s, last ? 1 : 0);
        if (!grid_barrier(e.bar, e.nblocks)) return;
        ib_phase(1, last ? 0 : 1, s == e.n_steps - 2);
        if (!last && !grid_barrier(e.bar, e.nblocks)) return;
    }
}

// The split schedule's lattice launch: one CTA per lattice item (nodes_per_item
// nodes of one tissue), the update of lbib_step's lattice kernel with its
// programmatic wait on the IB launch before it.  WIDE: two CTAs per SM fewer
// than the standalone kernel, for registers enough not to spill (at the
// standalone kernel's 40 registers with one species the update spills about
// 120 bytes: the tissue's arguments are read from shared memory, not from the
// constant bank).
template <int S, int FORCING, bool WIDE>
__global__ void __launch_bounds__(kLatticeThreads,
                                  LatticeOccupancy<float, S>::kMinBlocks - (WIDE ? 2 : 0))
    ens_lattice_kernel(EnsArgs e, int step, int out) {
    // the tissue's arguments in shared memory, read from there at each use
    // (held in registers they would spill at the standalone kernel's budget)
    __shared__ TissueDev td;
    const int item = blockIdx.x;
    const int t = find_tissue(e.item_pfx, e.n, item);
    {
        const int* src = reinterpret_cast<const int*>(e.tis + t);
        int* dst = reinterpret_cast<int*>(&td);
        for (int i = threadIdx.x; i < (int)(sizeof(TissueDev) / 4); i += kLatticeThreads)
            dst[i] = __ldg(src + i);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if ((td.cur + step) & 1) {
            const void* f0 = td.la.fsrc;
            td.la.fsrc = td.la.fdst;
            td.la.fdst = const_cast<void*>(f0);
            const void* g0 = td.la.gsrc;
            td.la.gsrc = td.la.gdst;
            td.la.gdst = const_cast<void*>(g0);
        }
        td.la.out = out;
    }
    __syncthreads();
    // node indices below 2^31 + nodes_per_item: unsigned 32-bit
    const unsigned nxr = (unsigned)td.nxr;
    const unsigned v0 = (unsigned)(item - e.item_pfx[t]) * (unsigned)e.nodes_per_item;
    for (int v = threadIdx.x; v < e.nodes_per_item; v += kLatticeThreads) {
        const unsigned vv = v0 + (unsigned)v;
        const unsigned yu = vv / nxr, xu = vv - yu * nxr;
        if (yu >= (unsigned)td.la.ny || xu >= (unsigned)td.la.nx) continue;
        const int x = (int)xu, y = (int)yu;
        if (td.bc_y)
            lattice_node<float, float, S, true, FORCING, false, true>(td.la, td.k, x, y);
        else
            lattice_node<float, float, S, false, FORCING, false, true>(td.la, td.k, x, y);
    }
}

// The split schedule's IB launch: one CTA of NT threads per cell of every
// tissue (move and/or prep as lbib_step's IB launch, with its programmatic
// wait on the lattice launch before it).
template <int NT>
__global__ void __launch_bounds__(NT) ens_ib_kernel(EnsArgs e, int move, int prep, int vforce) {
    extern __shared__ __align__(16) unsigned char ens_ib_smem[];
    const IBShared32 view = ib_shared32_view(ens_ib_smem, e.maxv);
    // the tissue's arguments in shared memory (a local copy would live on
    // the stack)
    __shared__ IBArgs ia;
    const int item = blockIdx.x;
    const int t = find_tissue(e.cell_pfx, e.n, item);
    {
        const int* src = reinterpret_cast<const int*>(&e.tis[t].ia);
        int* dst = reinterpret_cast<int*>(&ia);
        for (int i = threadIdx.x; i < (int)(sizeof(IBArgs) / 4); i += NT) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ia.do_move = move;
        ia.do_prep = prep;
        ia.write_vforce = vforce;
        ia.do_ids = vforce;
    }
    __syncthreads();
    ib_cell_f32<NT, true, false, false>(ia, item - e.cell_pfx[t], view, threadIdx.x, 0);
}

// A barrier that cannot complete (it waits for one CTA more than the grid
// has): used by lbib_ensemble_selftest_timeout() to exercise the bounded wait.
__global__ void barrier_timeout_kernel(unsigned* bar, unsigned nblocks) {
    grid_barrier(bar, nblocks);
}

typedef void (*EnsKernel)(EnsArgs);

static EnsKernel pick_kernel(int S, int forcing) {
    switch (S * 2 + (forcing ? 1 : 0)) {
        case 0: return ensemble_kernel<0, 0>;
        case 1: return ensemble_kernel<0, 1>;
        case 2: return ensemble_kernel<1, 0>;
        case 3: return ensemble_kernel<1, 1>;
        case 4: return ensemble_kernel<2, 0>;
        case 5: return ensemble_kernel<2, 1>;
        case 6: return ensemble_kernel<3, 0>;
        case 7: return ensemble_kernel<3, 1>;
        case 8: return ensemble_kernel<4, 0>;
        default: return ensemble_kernel<4, 1>;
    }
}

typedef void (*EnsLatticeKernel)(EnsArgs, int, int);

template <bool WIDE>
static EnsLatticeKernel pick_lattice_kernel_w(int S, int forcing) {
    switch (S * 2 + (forcing ? 1 : 0)) {
        case 0: return ens_lattice_kernel<0, 0, WIDE>;
        case 1: return ens_lattice_kernel<0, 1, WIDE>;
        case 2: return ens_lattice_kernel<1, 0, WIDE>;
        case 3: return ens_lattice_kernel<1, 1, WIDE>;
        case 4: return ens_lattice_kernel<2, 0, WIDE>;
        case 5: return ens_lattice_kernel<2, 1, WIDE>;
        case 6: return ens_lattice_kernel<3, 0, WIDE>;
        case 7: return ens_lattice_kernel<3, 1, WIDE>;
        case 8: return ens_lattice_kernel<4, 0, WIDE>;
        default: return ens_lattice_kernel<4, 1, WIDE>;
    }
}

static EnsLatticeKernel pick_lattice_kernel(int S, int forcing, bool wide) {
    return wide ? pick_lattice_kernel_w<true>(S, forcing) : pick_lattice_kernel_w<false>(S, forcing);
}

static uint64_t up256(uint64_t v) { return (v + 255) / 256 * 256; }

}  // namespace lbib

using namespace lbib;

struct lbib_ensemble {
    int n = 0;
    std::vector<lbib_ctx*> ctx;
    std::vector<uint64_t> off;  // workspace offset of each tissue
    char* ws = nullptr;
    uint64_t bytes = 0;
    cudaStream_t stream = nullptr;
    uint64_t tab_off = 0, ipfx_off = 0, cpfx_off = 0, bar_off = 0;
    int S = 0, forcing = 0;
    int nodes_per_item = 256;
    int blocks_per_sm = 0;  // 0 = as many as fit
    int max_blocks_per_sm = 0;
    int n_sms = 0;
    int maxv = 0;           // vertex slots per cell in shared memory (largest cell)
    int schedule = LBIB_ENS_PERSISTENT;
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    bool graph_ok = true;
    std::string err;
};

static thread_local std::string g_ens_err;

static int ens_fail(lbib_ensemble* e, int code, const std::string& msg) {
    if (e) e->err = msg;
    set_thread_error(code, msg);
    g_ens_err = msg;
    return code;
}

static void ens_drop_graphs(lbib_ensemble* e) {
    for (auto& kv : e->graphs) cudaGraphExecDestroy(kv.second);
    e->graphs.clear();
}

static uint64_t ens_region_bytes(int n) {
    return up256(sizeof(TissueDev) * (uint64_t)n) + 2 * up256(4 * (uint64_t)(n + 1)) + 256;
}

// Build the per-tissue table and prefix sums (host), upload them.
// Shared memory per CTA follows the largest cell of the ensemble; when it
// changes, the CTAs that fit per SM and the captured graphs change with it.
static cudaError_t ens_fit_cells(lbib_ensemble* e) {
    int mv = 8;
    for (auto* c : e->ctx) mv = std::max(mv, c->maxv_cell);
    mv = std::min((mv + 7) / 8 * 8, kMaxVertsPerCell);
    if (mv == e->maxv && e->max_blocks_per_sm > 0) return cudaSuccess;
    const size_t smem = (size_t)(kIBThreads / ens_cell_threads(mv)) * ens_cell_smem(mv);
    const void* k = (const void*)pick_kernel(e->S, e->forcing);
    cudaError_t er = cudaSuccess;
    if (smem > 48 * 1024)
        er = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (er == cudaSuccess)
        er = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kIBThreads, smem);
    if (er != cudaSuccess) return er;
    if (per < 1) return cudaErrorInvalidConfiguration;
    // the split schedule's IB kernel: one cell slot per CTA
    const size_t smem1 = ens_cell_smem(mv);
    if (smem1 > 48 * 1024) {
        er = ens_cell_threads(mv) == 64
                 ? cudaFuncSetAttribute((const void*)ens_ib_kernel<64>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1)
                 : cudaFuncSetAttribute((const void*)ens_ib_kernel<128>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
        if (er != cudaSuccess) return er;
    }
    ens_drop_graphs(e);
    e->maxv = mv;
    e->max_blocks_per_sm = per;
    return cudaSuccess;
}

static cudaError_t ens_upload(lbib_ensemble* e, int* total_items, int* total_cells) {
    cudaError_t fe = ens_fit_cells(e);
    if (fe != cudaSuccess) return fe;
    std::vector<TissueDev> tab((size_t)e->n);
    std::vector<int> ipfx((size_t)e->n + 1, 0), cpfx((size_t)e->n + 1, 0);
    // the tissues stream through one L2: their summed planes decide the
    // population load policy
    int64_t planes = 0;
    for (int t = 0; t < e->n; ++t) planes += e->ctx[t]->L.plane;
    const int l2_first =
        e->n > 0 && lattice_l2_first(LBIB_FP32, e->ctx[0]->p.n_species, planes) ? 1 : 0;
    for (int t = 0; t < e->n; ++t) {
        lbib_ctx* c = e->ctx[t];
        TissueDev& d = tab[t];
        std::memset(&d, 0, sizeof(d));
        d.la = ctx_lattice_args(c, 0, false);
        d.la.l2_first = l2_first;
        d.ia = ctx_ib_args(c, true, true, false);
        d.k = c->kf;
        d.bc_y = c->p.bc_y;
        d.nxr = (c->p.nx + 31) / 32 * 32;
        d.cur = c->cur;
        const int64_t nodes = (int64_t)d.nxr * c->p.ny;
        ipfx[t + 1] = ipfx[t] + (int)((nodes + e->nodes_per_item - 1) / e->nodes_per_item);
        cpfx[t + 1] = cpfx[t] + c->nC;
    }
    *total_items = ipfx[e->n];
    *total_cells = cpfx[e->n];
    cudaError_t er = cudaMemcpyAsync(e->ws + e->tab_off, tab.data(), sizeof(TissueDev) * e->n,
                                     cudaMemcpyHostToDevice, e->stream);
    if (er == cudaSuccess)
        er = cudaMemcpyAsync(e->ws + e->ipfx_off, ipfx.data(), 4 * (e->n + 1),
                             cudaMemcpyHostToDevice, e->stream);
    if (er == cudaSuccess)
        er = cudaMemcpyAsync(e->ws + e->cpfx_off, cpfx.data(), 4 * (e->n + 1),
                             cudaMemcpyHostToDevice, e->stream);
    if (er == cudaSuccess) er = cudaStreamSynchronize(e->stream);
    return er;
}

static EnsArgs ens_args(lbib_ensemble* e, int n_steps, int total_items, int total_cells,
                        unsigned nblocks) {
    EnsArgs a;
    a.tis = reinterpret_cast<const TissueDev*>(e->ws + e->tab_off);
    a.item_pfx = reinterpret_cast<const int*>(e->ws + e->ipfx_off);
    a.cell_pfx = reinterpret_cast<const int*>(e->ws + e->cpfx_off);
    a.n = e->n;
    a.n_steps = n_steps;
    a.nodes_per_item = e->nodes_per_item;
    a.total_items = total_items;
    a.total_cells = total_cells;
    a.bar = reinterpret_cast<unsigned*>(e->ws + e->bar_off);
    a.nblocks = nblocks;
    a.maxv = e->maxv;
    a.cell_threads = ens_cell_threads(e->maxv);
    return a;
}

static unsigned ens_grid(lbib_ensemble* e) {
    int per = e->blocks_per_sm > 0 ? std::min(e->blocks_per_sm, e->max_blocks_per_sm)
                                   : e->max_blocks_per_sm;
    if (per < 1) per = 1;
    return (unsigned)(per * e->n_sms);
}

static cudaError_t ens_launch(lbib_ensemble* e, const EnsArgs& a, unsigned grid,
                              cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kIBThreads);
    cfg.dynamicSmemBytes = (size_t)(kIBThreads / a.cell_threads) * ens_cell_smem(a.maxv);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pick_kernel(e->S, e->forcing), a);
}

// The split schedule of n steps: the prep, then per step the lattice launch
// and the IB launch (move, and the prep of the next step but after the last).
// Every launch after the first is programmatic; without cells the lattice
// launches follow one another and wait for each other in full.
static cudaError_t ens_split_enqueue(lbib_ensemble* e, const EnsArgs& a, cudaStream_t st) {
    const size_t smem = ens_cell_smem(a.maxv);
    auto ib = [&](int move, int prep, int vforce, bool pdl) -> cudaError_t {
        if (a.total_cells == 0) return cudaSuccess;
        if (a.cell_threads == 64)
            return launch_kernel(ens_ib_kernel<64>, dim3(a.total_cells), dim3(64), smem, st, pdl,
                                 a, move, prep, vforce);
        return launch_kernel(ens_ib_kernel<128>, dim3(a.total_cells), dim3(128), smem, st, pdl, a,
                             move, prep, vforce);
    };
    const EnsLatticeKernel lk =
        pick_lattice_kernel(e->S, e->forcing, e->schedule == LBIB_ENS_SPLIT_WIDE);
    const bool pdl = a.total_cells > 0;
    cudaError_t er = ib(0, 1, a.n_steps == 1, false);
    for (int s = 0; s < a.n_steps && er == cudaSuccess; ++s) {
        const bool last = (s == a.n_steps - 1);
        er = launch_kernel(lk, dim3(a.total_items), dim3(kLatticeThreads), 0, st, pdl, a, s,
                           last ? 1 : 0);
        if (er == cudaSuccess) er = ib(1, last ? 0 : 1, s == a.n_steps - 2, true);
    }
    return er;
}

static cudaError_t ens_enqueue(lbib_ensemble* e, const EnsArgs& a, unsigned grid,
                               cudaStream_t st) {
    return e->schedule == LBIB_ENS_PERSISTENT ? ens_launch(e, a, grid, st)
                                              : ens_split_enqueue(e, a, st);
}

extern "C" {

int lbib_ensemble_workspace_size(int32_t n, const lbib_params* params,
                                 const int32_t* max_vertices, const int32_t* max_cells,
                                 uint64_t* bytes_out) {
    if (n < 1 || !params || !max_vertices || !max_cells || !bytes_out)
        return ens_fail(nullptr, LBIB_E_PARAM, "lbib_ensemble_workspace_size: invalid arguments");
    uint64_t total = 0;
    for (int t = 0; t < n; ++t) {
        uint64_t b = 0;
        int rc = lbib_workspace_size(params + t, max_vertices[t], max_cells[t], &b);
        if (rc) return rc;
        total += up256(b);
    }
    *bytes_out = total + ens_region_bytes(n);
    return LBIB_OK;
}

int lbib_ensemble_create(int32_t n, const lbib_params* params, const int32_t* max_vertices,
                         const int32_t* max_cells, void* d_workspace, uint64_t bytes,
                         void* cuda_stream, lbib_ensemble** out) {
    if (!out) return ens_fail(nullptr, LBIB_E_PARAM, "out is NULL");
    *out = nullptr;
    uint64_t need = 0;
    int rc = lbib_ensemble_workspace_size(n, params, max_vertices, max_cells, &need);
    if (rc) return rc;
    for (int t = 0; t < n; ++t) {
        if (params[t].precision != LBIB_FP32)
            return ens_fail(nullptr, LBIB_E_PARAM, "ensemble tissues use FP32 storage");
        if (params[t].junction_period > 0)
            return ens_fail(nullptr, LBIB_E_PARAM,
                            "ensemble tissues have no cell junctions (they need separate launches)");
        if (params[t].noflux_mask || params[t].mass_sources || params[t].pressure_nodes ||
            params[t].node_sources)
            return ens_fail(nullptr, LBIB_E_PARAM,
                            "ensemble tissues have no domain planes, mass sources or pressure nodes");
        if (params[t].n_species != params[0].n_species || params[t].forcing != params[0].forcing)
            return ens_fail(nullptr, LBIB_E_PARAM,
                            "ensemble tissues share the species count and forcing");
    }
    if (!d_workspace || bytes < need || reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return ens_fail(nullptr, LBIB_E_WORKSPACE,
                        "ensemble workspace NULL, misaligned or smaller than " +
                            std::to_string(need));
    lbib_ensemble* e = new (std::nothrow) lbib_ensemble();
    if (!e) return ens_fail(nullptr, LBIB_E_PARAM, "out of host memory");
    e->n = n;
    e->ws = static_cast<char*>(d_workspace);
    e->bytes = bytes;
    e->stream = static_cast<cudaStream_t>(cuda_stream);
    e->S = params[0].n_species;
    e->forcing = params[0].forcing;
    uint64_t o = 0;
    for (int t = 0; t < n; ++t) {
        uint64_t b = 0;
        lbib_workspace_size(params + t, max_vertices[t], max_cells[t], &b);
        lbib_ctx* c = nullptr;
        rc = lbib_create(params + t, max_vertices[t], max_cells[t], e->ws + o, b, cuda_stream, &c);
        if (rc) {
            for (auto* x : e->ctx) lbib_destroy(x);
            delete e;
            return rc;
        }
        e->ctx.push_back(c);
        e->off.push_back(o);
        o += up256(b);
    }
    e->tab_off = o;
    e->ipfx_off = e->tab_off + up256(sizeof(TissueDev) * (uint64_t)n);
    e->cpfx_off = e->ipfx_off + up256(4 * (uint64_t)(n + 1));
    e->bar_off = e->cpfx_off + up256(4 * (uint64_t)(n + 1));
    int dev = 0;
    cudaError_t er = cudaGetDevice(&dev);
    if (er == cudaSuccess) er = cudaDeviceGetAttribute(&e->n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (er == cudaSuccess) er = ens_fit_cells(e);
    if (er == cudaSuccess) er = cudaMemsetAsync(e->ws + e->bar_off, 0, 256, e->stream);
    if (er == cudaSuccess) er = cudaStreamSynchronize(e->stream);
    if (er != cudaSuccess || e->max_blocks_per_sm < 1) {
        for (auto* x : e->ctx) lbib_destroy(x);
        delete e;
        return ens_fail(nullptr, LBIB_E_CUDA,
                        std::string("lbib_ensemble_create: ") + cudaGetErrorString(er));
    }
    *out = e;
    return LBIB_OK;
}

lbib_ctx* lbib_ensemble_tissue(lbib_ensemble* e, int32_t t) {
    if (!e || t < 0 || t >= e->n) return nullptr;
    return e->ctx[t];
}

int lbib_ensemble_step(lbib_ensemble* e, int32_t n_steps) {
    NvtxRange nvtx_range("lbib_ensemble_step");
    if (!e) return LBIB_E_PARAM;
    if (n_steps < 0) return ens_fail(e, LBIB_E_PARAM, "n_steps must be >= 0");
    if (n_steps == 0) return LBIB_OK;
    int items = 0, cells = 0;
    cudaError_t er = ens_upload(e, &items, &cells);
    // a tissue's pending asynchronous readback ends before its cells move
    for (auto* c : e->ctx)
        if (er == cudaSuccess) er = rb_fence(c, e->stream);
    if (er != cudaSuccess)
        return ens_fail(e, LBIB_E_CUDA, std::string("lbib_ensemble_step: ") + cudaGetErrorString(er));
    const unsigned grid = ens_grid(e);
    const EnsArgs a = ens_args(e, n_steps, items, cells, grid);
    // the kernel reads the table at run time; the graph depends only on the
    // step count, the launch shape and the work totals
    const auto key = std::make_tuple((int)n_steps, items, cells);
    auto it = e->graphs.find(key);
    bool launched = false;
    if (e->graph_ok && it == e->graphs.end()) {
        cudaStream_t cap;
        er = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        cudaGraph_t g = nullptr;
        if (er == cudaSuccess) er = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (er == cudaSuccess) {
            cudaError_t e2 = ens_enqueue(e, a, grid, cap);
            er = cudaStreamEndCapture(cap, &g);
            if (e2 != cudaSuccess) er = e2;
        }
        cudaGraphExec_t ex = nullptr;
        if (er == cudaSuccess) er = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (er == cudaSuccess) {
            it = e->graphs.emplace(key, ex).first;
        } else {
            cudaGetLastError();
            e->graph_ok = false;  // fall back to direct launches
        }
    }
    if (e->graph_ok && it != e->graphs.end()) {
        er = cudaGraphLaunch(it->second, e->stream);
        launched = true;
    }
    if (!launched) er = ens_enqueue(e, a, grid, e->stream);
    if (er != cudaSuccess)
        return ens_fail(e, LBIB_E_CUDA, std::string("lbib_ensemble_step: ") + cudaGetErrorString(er));
    for (auto* c : e->ctx) {
        c->cur = (c->cur + n_steps) & 1;
        c->fields_valid = true;
        c->vforce_valid = c->nC > 0;
    }
    return LBIB_OK;
}

int lbib_ensemble_status(lbib_ensemble* e) {
    if (!e) return LBIB_E_PARAM;
    unsigned bar[3] = {0, 0, 0};
    cudaError_t er = cudaMemcpyAsync(bar, e->ws + e->bar_off, sizeof(bar), cudaMemcpyDeviceToHost,
                                     e->stream);
    if (er == cudaSuccess) er = cudaStreamSynchronize(e->stream);
    if (er != cudaSuccess)
        return ens_fail(e, LBIB_E_CUDA, std::string("lbib_ensemble_status: ") + cudaGetErrorString(er));
    if (bar[2]) {
        // clear the barrier state so that the ensemble can run again
        cudaMemsetAsync(e->ws + e->bar_off, 0, 256, e->stream);
        cudaStreamSynchronize(e->stream);
        return ens_fail(e, LBIB_E_TIMEOUT, "a grid barrier wait ran out (about one second)");
    }
    return LBIB_OK;
}

int lbib_ensemble_config(lbib_ensemble* e, int32_t nodes_per_item, int32_t blocks_per_sm,
                         int32_t* graph_out, int32_t* grid_out) {
    if (!e) return LBIB_E_PARAM;
    if (nodes_per_item > 0) {
        if (nodes_per_item % kIBThreads)
            return ens_fail(e, LBIB_E_PARAM, "nodes_per_item must be a multiple of 256");
        if (nodes_per_item != e->nodes_per_item) ens_drop_graphs(e);
        e->nodes_per_item = nodes_per_item;
    }
    if (blocks_per_sm >= 0) {
        if (blocks_per_sm != e->blocks_per_sm) ens_drop_graphs(e);
        e->blocks_per_sm = blocks_per_sm;
    }
    if (graph_out) *graph_out = e->graph_ok ? 1 : 0;
    if (grid_out) *grid_out = (int32_t)ens_grid(e);
    return LBIB_OK;
}

int lbib_ensemble_schedule(lbib_ensemble* e, int32_t schedule, int32_t* schedule_out) {
    if (!e) return LBIB_E_PARAM;
    if (schedule >= 0) {
        if (schedule != LBIB_ENS_PERSISTENT && schedule != LBIB_ENS_SPLIT &&
            schedule != LBIB_ENS_SPLIT_WIDE)
            return ens_fail(e, LBIB_E_PARAM,
                            "schedule must be LBIB_ENS_PERSISTENT, LBIB_ENS_SPLIT or "
                            "LBIB_ENS_SPLIT_WIDE");
        if (schedule != e->schedule) ens_drop_graphs(e);
        e->schedule = schedule;
    }
    if (schedule_out) *schedule_out = e->schedule;
    return LBIB_OK;
}

int lbib_ensemble_tune(lbib_ensemble* e, int32_t trial_steps, int32_t* config_out,
                       double* ms_out) {
    if (!e || trial_steps < 1 || !config_out) return LBIB_E_PARAM;
    const int npis[5] = {256, 512, 1024, 2048, 4096};
    double best = 1e300;
    int best_npi = e->nodes_per_item, best_bps = e->blocks_per_sm, best_sched = e->schedule;
    double best_p = 1e300;  // the persistent kernel's best, whose CTAs per SM are kept
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    for (int npi : npis) {
        // bps 1..max: the persistent kernel; bps -1 and 0: the split
        // schedule (-1 its wide lattice kernel)
        for (int bps = -1; bps <= e->max_blocks_per_sm; ++bps) {
            e->nodes_per_item = npi;
            e->schedule = bps > 0 ? LBIB_ENS_PERSISTENT
                                  : (bps == 0 ? LBIB_ENS_SPLIT : LBIB_ENS_SPLIT_WIDE);
            e->blocks_per_sm = bps > 0 ? bps : 1;
            int items = 0, cells = 0;
            cudaError_t er = ens_upload(e, &items, &cells);
            const unsigned grid = ens_grid(e);
            const EnsArgs a = ens_args(e, trial_steps, items, cells, grid);
            float ms = 0.f, msb = 1e30f;
            for (int rep = 0; rep < 2 && er == cudaSuccess; ++rep) {
                er = cudaEventRecord(t0, e->stream);
                if (er == cudaSuccess) er = ens_enqueue(e, a, grid, e->stream);
                if (er == cudaSuccess) er = cudaEventRecord(t1, e->stream);
                if (er == cudaSuccess) er = cudaEventSynchronize(t1);
                if (er == cudaSuccess) er = cudaEventElapsedTime(&ms, t0, t1);
                for (auto* c : e->ctx) c->cur = (c->cur + trial_steps) & 1;
                if (er == cudaSuccess) msb = std::min(msb, ms);
            }
            if (er != cudaSuccess) {
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
                return ens_fail(e, LBIB_E_CUDA, std::string("lbib_ensemble_tune: ") +
                                                    cudaGetErrorString(er));
            }
            const int st = lbib_ensemble_status(e);
            if (st) {
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
                return st;
            }
            if (msb < best) {
                best = msb;
                best_npi = npi;
                best_sched = e->schedule;
            }
            if (bps > 0 && msb < best_p) {
                best_p = msb;
                best_bps = bps;
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (auto* c : e->ctx) {
        c->fields_valid = true;
        c->vforce_valid = c->nC > 0;
    }
    ens_drop_graphs(e);
    e->nodes_per_item = best_npi;
    e->blocks_per_sm = best_bps;
    e->schedule = best_sched;
    config_out[0] = best_npi;
    config_out[1] = best_bps;
    if (ms_out) *ms_out = best / trial_steps;
    return LBIB_OK;
}

int lbib_ensemble_selftest_timeout(lbib_ensemble* e, double* seconds_out) {
    if (!e) return LBIB_E_PARAM;
    unsigned* bar = reinterpret_cast<unsigned*>(e->ws + e->bar_off);
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cudaError_t er = cudaMemsetAsync(bar, 0, 256, e->stream);
    if (er == cudaSuccess) er = cudaEventRecord(t0, e->stream);
    if (er == cudaSuccess) {
        barrier_timeout_kernel<<<1, 32, 0, e->stream>>>(bar, 2u);  // waits for a CTA that never comes
        er = cudaGetLastError();
    }
    if (er == cudaSuccess) er = cudaEventRecord(t1, e->stream);
    if (er == cudaSuccess) er = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (er == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (er != cudaSuccess)
        return ens_fail(e, LBIB_E_CUDA, std::string("selftest: ") + cudaGetErrorString(er));
    if (seconds_out) *seconds_out = ms * 1e-3;
    return lbib_ensemble_status(e);
}

void lbib_ensemble_destroy(lbib_ensemble* e) {
    if (!e) return;
    ens_drop_graphs(e);
    for (auto* c : e->ctx) lbib_destroy(c);
    delete e;
}

const char* lbib_ensemble_last_error(const lbib_ensemble* e) {
    return e ? e->err.c_str() : g_ens_err.c_str();
}

}  // extern "C"
