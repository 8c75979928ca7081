// lbib_internal.cuh -- structures shared by the CUDA translation units of the
// coupled LB-IB library (not part of the public ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#ifndef LBIB_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif
#include <stdint.h>

#include <cmath>
#include <string>

#include "../../include/lbib.h"

namespace lbib {

// A named NVTX range over a host call: a profiler's timeline shows each as a
// span around the launches (or graph launches) it enqueues; without an
// attached tool a push or pop is a test of one function pointer.  Building
// with -DLBIB_NO_NVTX removes them.
struct NvtxRange {
    explicit NvtxRange(const char* name) {
#ifndef LBIB_NO_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange() {
#ifndef LBIB_NO_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// D2Q9 velocity set in the order v0 = 0, v1..v4 = axes (cos, sin)(pi(i-1)/2),
// v5..v8 = diagonals (1,1), (-1,1), (-1,-1), (1,-1)  (Sec. 6.1 footnotes).
// D2Q5 uses v0..v4.  Weights: D2Q9 4/9, 1/9, 1/36; D2Q5 1/3, 1/6.
__host__ __device__ constexpr int cx(int q) {
    return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int q) {
    return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int q) {
    return q == 0 ? 0 : (q <= 4 ? ((q + 1) % 4) + 1 : ((q - 5 + 2) % 4) + 5);
}
__host__ __device__ constexpr double w9(int q) {
    return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr double w5(int q) { return q == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }

constexpr int kMaxSpecies = 4;
constexpr int kMaxVertsPerCell = 1024;  // vertices of one cell held in shared memory
constexpr int kMaxRows = 128;           // scanline rows per cell (else brute force)
constexpr int kMaxCross = 8;            // crossings per scanline row (else brute force)
constexpr uint32_t kOutside = 0xFFFFFFFFu;

// Bits of the 16-bit no-flux closure code of a node (direction q = 1..4 of
// D2Q5): the population arriving along v_q comes from another domain (not a
// wall link); x + v_q lies in the node's domain; x + 2 v_q does too; some
// closure reads this node's moments.
constexpr int kNcodeMiss = 0;    // bits 0..3
constexpr int kNcodeIn1 = 4;     // bits 4..7
constexpr int kNcodeIn2 = 8;     // bits 8..11
constexpr int kNcodeMom = 12;    // bit 12

// diagnostic words at the start of the diag region
enum Diag : int {
    kDiagNonFinite = 0,   // a non-finite rho or u was produced
    kDiagWallStencil = 1, // an IB stencil node fell outside a walled domain (dropped)
    kDiagRasterSlow = 2,  // a cell used the brute-force labelling path
    kDiagGeometry = 3,    // a cell's bounding box became non-finite or wider than the lattice
    kDiagCheck = 4,       // checking build: an access failed its bounds or alignment check
    kDiagCheckSite = 5,   // checking build: site of the first failed check (CheckSite)
    kDiagCheckAddr = 6,   // checking build: low 32 bits of its address
    kDiagWords = 64
};

// Sites of the checking build's access checks (kDiagCheckSite).
enum CheckSite : uint32_t {
    kSiteLatticeIndex = 1,  // a pulled population's index outside the plane
    kSiteLatticeAlign = 2,  // a plane base not aligned to its element
    kSiteClosureIndex = 3,  // a no-flux closure's moment index outside the plane
    kSitePairIndex = 4,     // FP16 pair kernel: a word index outside the plane
    kSitePairAlign = 5,     // FP16 pair kernel: a 16-byte access not aligned
    kSiteMask = 6,          // a group-mask word outside the mask
    kSiteIbVertex = 7,      // a vertex index outside the vertex arrays
    kSiteIbU = 8,           // an interpolation load outside the velocity plane or misaligned
    kSiteIbForce = 9,       // a spreading reduction outside the force plane or misaligned
    kSiteIbLabel = 10,      // a label or source write outside its plane or misaligned
    kSiteIbShared = 11,     // a vertex slot outside the cell's shared arrays
};

// The checking build (compiled with -DLBIB_CHECK into a library of its own):
// the kernels test the address of every access that needs an alignment or
// could leave its array, and an access that fails is skipped (a load reads
// zero) after the first failure's site and address are recorded in the diag
// words.  Nothing traps.  The plain build compiles every check to `true`.
#ifdef LBIB_CHECK
__device__ __noinline__ inline void check_failed(uint32_t* diag, uint32_t site, const void* p) {
    if (!diag) return;
    if (atomicOr(diag + kDiagCheck, 1u) == 0u) {
        atomicExch(diag + kDiagCheckSite, site);
        atomicExch(diag + kDiagCheckAddr, (uint32_t)reinterpret_cast<uintptr_t>(p));
    }
}
// p: the access of `bytes` bytes (aligned to `bytes`), inside [lo, hi) when
// lo is given
__device__ __forceinline__ bool check_access(uint32_t* diag, uint32_t site, const void* p,
                                             int bytes, const void* lo, const void* hi) {
    const char* c = static_cast<const char*>(p);
    bool ok = (reinterpret_cast<uintptr_t>(p) & (uintptr_t)(bytes - 1)) == 0;
    if (lo && (c < static_cast<const char*>(lo) || c + bytes > static_cast<const char*>(hi)))
        ok = false;
    if (!ok) check_failed(diag, site, p);
    return ok;
}
// an index of an array of n elements
__device__ __forceinline__ bool check_index(uint32_t* diag, uint32_t site, int64_t i, int64_t n) {
    const bool ok = i >= 0 && i < n;
    if (!ok) check_failed(diag, site, reinterpret_cast<const void*>(i));
    return ok;
}
#define LBIB_CHK_ACCESS(diag, site, p, bytes, lo, hi) \
    ::lbib::check_access((diag), (site), (p), (bytes), (lo), (hi))
#define LBIB_CHK_INDEX(diag, site, i, n) ::lbib::check_index((diag), (site), (i), (n))
#else
#define LBIB_CHK_ACCESS(diag, site, p, bytes, lo, hi) true
#define LBIB_CHK_INDEX(diag, site, i, n) true
#endif

// Workspace layout: byte offsets into the caller's device workspace.
struct Layout {
    int64_t pitch = 0;         // elements per lattice row
    int64_t plane = 0;         // elements per plane (pitch * ny)
    int es = 0, cs = 0;        // storage / compute element bytes
    uint64_t f[2] = {0, 0}, g[2] = {0, 0};
    uint64_t force = 0, u = 0, rho = 0, phi = 0, id = 0, id_out = 0, force_out = 0;
    uint64_t xy = 0, L0 = 0, k = 0, vforce = 0, off = 0, pres = 0, srcf = 0, area = 0;
    uint64_t vbase = 0, vfrac = 0, fmask = 0, lmask = 0, src = 0, smask = 0;
    uint64_t dom = 0;          // domain labels of the confined species (noflux_mask != 0)
    // the no-flux closure of Sec. 6.1 (noflux_scheme 0): a 16-bit code per
    // node (kNcode* bits) and the species moments (phi, jx, jy per species,
    // compute type, plane stride `plane`) of the previous step, by parity
    uint64_t ncode = 0, mom[2] = {0, 0};
    // cell junctions (junction_period > 0): partner and cell of every vertex, bins
    uint64_t jpartner = 0, jcell = 0, jcnt = 0, jstart = 0, jvbin = 0, jent = 0;
    uint64_t mrate = 0, marea = 0, msrc = 0;  // per-cell mass source data (mass_sources)
    uint64_t pnode = 0;        // internal pressure nodes, one byte per node (pressure_nodes)
    uint64_t nsrc = 0;         // static mass source per node, compute type (node_sources)
    int jnbx = 0, jnby = 0;
    // FP64 conservation sums (lbib_get_sums): global, per cell, non-finite count
    uint64_t sums = 0, sums_bytes = 0;
    uint64_t diag = 0;
    uint64_t total = 0;
};

bool make_layout(const lbib_params& p, int max_vertices, int max_cells, Layout* L);

// Coefficients of the lattice update, in the compute type.
template <typename C>
struct Coefs {
    C rho0, omega, pref;        // 1/tau, 1 - 1/(2 tau) (Guo)
    C bfx, bfy;                 // uniform body force density
    C omegaD[kMaxSpecies];      // 1/tau_D
    C K[kMaxSpecies][kMaxSpecies];  // react - diag(decay)
    C srate[kMaxSpecies];
    C fscale[9], finv[9];       // stored = (f - w rho0) * finv; dev = stored * fscale
    C gscale[5], ginv[5];
    C omc;                      // 1 - omega
    C omcD[kMaxSpecies];        // 1 - omega_D
    C isig, isig_g;             // 1/sigma, 1/sigma_g of scaled (FP16) storage, else 1
    int react_model;            // LBIB_REACT_LINEAR or LBIB_REACT_SCHNAKENBERG
    C sgamma, sa, sb;           // Schnakenberg gamma, a, b
    C prho;                     // density held at internal pressure nodes
    // lattice weights in the compute type.  D2Q5 (rest, axes): a pair that
    // sums to one exactly in that type, so the species update creates no mass
    // from their rounding (with the nearest FP32 values of 1/3 and 1/6 every
    // update added 3e-8 of the species' mass, 1.7e-5 of the concentration
    // over 2000 steps of the 512^2 tissue, 2.0e-6 with these).  D2Q9 (rest,
    // axes, diagonals): the nearest values; the fluid is stored as deviations
    // from rest, which keeps their rounding small, and moving the diagonal
    // weight off its nearest value to make the FP32 sum exact raised the
    // FP32 velocity error at 2000 steps from 7.9e-5 to 1.3e-4.
    C w9c[3];
    C w5c[2];
};

// The weight sets of Coefs::w9c / w5c for the compute type C (FP64: both
// sets sum to one exactly as computed).
template <typename C>
inline void exact_sum_weights(C w9c[3], C w5c[2]);
template <>
inline void exact_sum_weights<double>(double w9c[3], double w5c[2]) {
    w9c[1] = 1.0 / 9.0;
    w9c[2] = 1.0 / 36.0;
    w9c[0] = 1.0 - 4.0 * w9c[1] - 4.0 * w9c[2];
    w5c[1] = 1.0 / 6.0;
    w5c[0] = 1.0 - 4.0 * w5c[1];
}
template <>
inline void exact_sum_weights<float>(float w9c[3], float w5c[2]) {
    w9c[0] = (float)(4.0 / 9.0);
    w9c[1] = (float)(1.0 / 9.0);
    w9c[2] = (float)(1.0 / 36.0);
    // 1 - 4 w1 is exact in FP32 (Sterbenz): the pair sums to one exactly
    w5c[1] = (float)(1.0 / 6.0);
    w5c[0] = 1.0f - 4.0f * w5c[1];
}

struct LatticeArgs {
    const void* fsrc;
    void* fdst;
    const void* gsrc;
    void* gdst;
    void* force;        // interleaved (fx, fy) per node, compute type; read then cleared
    uint32_t* id;       // packed labels (cell << 4 | src bits), kOutside = none; read then
                        // cleared (written by the IB prep of an output step only); may be NULL
    uint8_t* src;       // source bits of the node (OR over the cells containing it), one
                        // byte per node; read then cleared
    void* u;            // interleaved (ux, uy) per node, compute type (written)
    void* rho;          // written when out
    void* phi;          // S planes, written when out
    uint32_t* id_out;   // written when out
    void* force_out;    // written when out
    uint32_t* diag;
    int nx, ny;
    int64_t pitch, plane;
    int out;            // write rho, phi, id_out, force_out
    int ib;             // read/clear force and labels
    int l2_first;       // population loads evict-first in L2 (else normal)
    const int32_t* dom; // domain label per node (pitch layout), NULL = none
    int noflux;         // bit s: species s is confined to its domain
    // the no-flux closure (Sec. 6.1) of the confined species: the node codes
    // (NULL: half-way bounce-back on the links between domains instead), the
    // moments of the previous step (read at the closures) and of this step
    // (written where the code asks for them); 3 planes per species
    const uint16_t* ncode;
    const void* mom_in;
    void* mom_out;
    // 1 bit per 4 consecutive nodes (node index >> 2): groups that received
    // spread force / labels / source bits this step.  fmask NULL = dense
    // (read every node).
    uint32_t* fmask;
    uint32_t* lmask;
    uint32_t* smask;
    // mass sources (Sec. 3.2.3): S_c of every cell for this step (compute
    // type, written by the IB prep), added at the nodes labelled c; NULL = none
    const void* msrc;
    // internal pressure nodes (Sec. 6.1): one byte per node (pitch layout),
    // nonzero = populations rescaled to the density prho; NULL = none
    const uint8_t* pnode;
    // static mass source per node (compute type, pitch layout), added to the
    // cell's; NULL = none
    const void* nsrc;
};

struct IBArgs {
    double2* xy;
    const double* L0;
    const double* k;
    const int32_t* off;
    const double* pres;
    const uint8_t* srcf;
    double2* vforce;
    void* force;
    uint32_t* id;
    const void* u;
    uint32_t* diag;
    int nx, ny, bc_y, n_cells;
    int64_t pitch;
    int64_t plane;      // elements per plane of the force / u / label / source planes
    double tension;
    int do_move, do_prep, do_mask, write_vforce;
    int do_force;       // compute and spread vertex forces (0: labels only)
    int2* vbase;        // FP32 path, optional: floor(X) per vertex handed to the next move
    float2* vfrac;      // FP32 path, optional: X - floor(X) per vertex
    uint32_t* fmask;    // optional: mark the groups that receive spread force
    uint32_t* lmask;    // optional: mark the groups that receive labels
    void* src;          // optional source-bits plane (OR of the cells' bits): one byte per
                        // node, rows 8-byte aligned; with src_words one uint32 per node
    uint32_t* smask;    // optional: mark the groups that receive source bits
    int do_ids;         // write the packed labels into `id` (else only source bits)
    int src_words;
    // cell junctions (Eq. celljunctionforce): the partner vertex of each
    // vertex (-1 none), NULL = no junctions; spring constant, rest length, cutoff
    const int32_t* jpartner;
    double jk, jl0, jlmax;
    // mass sources (Sec. 3.2.3): the prep writes S_c = mrate[c] +
    // malpha (marea[c] - A_c) (A_c the polygon area after the move; without
    // marea S_c = mrate[c]) to msrc_out[c] in the lattice compute type; NULL = none
    void* msrc_out;
    const double* mrate;
    const double* marea;
    double malpha;
};

// Junction renewal: the vertices sorted into a uniform grid of bins at least
// l_max wide, CSR (count per bin, offsets, entries grouped by bin)
struct __align__(16) JunctionEntry {
    float x, y;  // wrapped position in FP32 (for the prefilter)
    int cell, v;
};
struct JunctionArgs {
    const double2* xy;
    const int32_t* vcell;   // cell index of every vertex
    int32_t* partner;
    int* cnt;               // nbins: counts, then fill cursors
    int* start;             // nbins + 1 offsets into ent
    int* vbin;              // bin of every vertex
    JunctionEntry* ent;     // nv entries
    int nv, nx, ny, bc_y, nbx, nby;
    double inv_nx, inv_ny, inv_wbx, inv_wby, lmax;
    float fthr;             // FP32 prefilter bound on the squared distance
};

// The periodic minimum image d - n round(d/n) of a coordinate difference in
// FP64, with that expression's result: for |d| <= 0.49 n the quotient rounds
// to zero and d comes back unchanged, so the division (slow at this GPU's
// FP64 rate) only runs for differences across the periodic seam.
__device__ __forceinline__ double min_image(double d, int n) {
    if (fabs(d) <= 0.49 * (double)n) return d;
    return __dsub_rn(d, __dmul_rn((double)n, round(__ddiv_rn(d, (double)n))));
}

// shared memory of the FP32 per-cell IB work (one CTA per cell), as pointers
// into the CTA's shared memory; the vertex arrays hold `maxv` entries
struct IBShared32 {
    double2* sx;  // FP64 positions (exact fallbacks)
    int2* sb;     // floor(X)
    float2* sf;   // X - floor(X)
    int* rowcnt;  // kMaxRows
    int* thr;     // kMaxRows * kMaxCross
    int* sbox;    // 4
    int* s_flag;  // 1
    // the cell's force-mask words (kMaskTable keys and bits): the spreading
    // ORs its group bits here and the CTA then ORs each distinct word into
    // the mask once
    uint32_t* mkey;
    uint32_t* mval;
    int maxv;
};

constexpr int kMaskTableLog2 = 8;
constexpr int kMaskTable = 1 << kMaskTableLog2;
constexpr uint32_t kMaskEmpty = 0xFFFFFFFFu;

// fixed part of the FP32 IB kernel's dynamic shared memory (bytes, 16-aligned)
constexpr int kIBSmemFixed =
    ((kMaxRows + kMaxRows * kMaxCross + 4 + 1 + 2 * kMaskTable) * 4 + 15) / 16 * 16;
constexpr int kIBSmemPerVertex = 16 + 8 + 8;

// the views of one cell slot of that shared memory (fixed part, then maxv
// vertices)
__device__ __forceinline__ IBShared32 ib_shared32_view(unsigned char* base, int maxv) {
    IBShared32 v;
    int* fixed = reinterpret_cast<int*>(base);
    v.rowcnt = fixed;
    v.thr = fixed + kMaxRows;
    v.sbox = v.thr + kMaxRows * kMaxCross;
    v.s_flag = v.sbox + 4;
    v.mkey = reinterpret_cast<uint32_t*>(v.s_flag + 1);
    v.mval = v.mkey + kMaskTable;
    v.sx = reinterpret_cast<double2*>(base + kIBSmemFixed);
    v.sb = reinterpret_cast<int2*>(v.sx + maxv);
    v.sf = reinterpret_cast<float2*>(v.sb + maxv);
    v.maxv = maxv;
    return v;
}

// a static shared-memory block for the largest cells (the persistent kernel)
struct IBSmem32 {
    double2 sx[kMaxVertsPerCell];  // FP64 positions (exact fallbacks)
    int2 sb[kMaxVertsPerCell];     // floor(X)
    float2 sf[kMaxVertsPerCell];   // X - floor(X)
    int rowcnt[kMaxRows];
    int thr[kMaxRows * kMaxCross];
    int sbox[4];
    int s_flag;
};

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream-serialization attribute may start while the previous kernel of its
// stream is still running.  griddep_wait() blocks the calling thread until
// that kernel has completed and its writes are visible;
// griddep_launch_dependents() lets the next such kernel of the stream start
// once every CTA of this grid has issued it or exited.  Both are no-ops for a
// kernel launched without the attribute.  Kernels of the coupled step call
// them in this order, so a kernel starts only after the kernel two launches
// back has completed: before its wait it may read what that kernel (or any
// earlier one) wrote, through L2 (`ld.global.cg`), and nothing else.
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// L2 eviction priorities (createpolicy).  The velocity and force planes near
// the membranes, which the lattice update writes and the IB kernel reads and
// accumulates right after (and the other way round), go last, so that they
// stay in L2 while the population streams pass through.  The population
// loads go first when both population buffers nearly fit in L2 (the lines
// just read are dead, so the ones just written survive to the next step:
// 1024^2 FP32 lattice launch 31.0 -> 28.9 us with both hints); on a lattice
// many times larger than L2 they stay normal (there evict-first cost 7%: a
// line shared by two warps can leave between their reads).
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_evict_normal() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// L2-only loads of the population streams under policy pol
__device__ __forceinline__ float ld_stream(const float* p, uint64_t pol) {
    float v;
    asm volatile("ld.global.cg.L2::cache_hint.f32 %0, [%1], %2;"
                 : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* p, uint64_t pol) {
    double v;
    asm volatile("ld.global.cg.L2::cache_hint.f64 %0, [%1], %2;"
                 : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ unsigned short ld_stream(const unsigned short* p, uint64_t pol) {
    unsigned short v;
    asm volatile("ld.global.cg.L2::cache_hint.b16 %0, [%1], %2;"
                 : "=h"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.cg.L2::cache_hint.b32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// stores of the velocity / force planes near the membranes, evict-last
__device__ __forceinline__ void st_keep(float2* p, float2 v) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "l"(l2_evict_last()) : "memory");
}
__device__ __forceinline__ void st_keep(double2* p, double2 v) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;"
                 :: "l"(p), "d"(v.x), "d"(v.y), "l"(l2_evict_last()) : "memory");
}
__device__ __forceinline__ void st_keep(float4* p, float4 v) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(l2_evict_last())
                 : "memory");
}
// accumulation into the force plane, evict-last: one node (8 bytes) or two
// adjacent nodes (16 bytes, p 16-byte aligned) per operation
__device__ __forceinline__ void red_keep(float2* p, float x, float y) {
    asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 :: "l"(p), "f"(x), "f"(y), "l"(l2_evict_last()) : "memory");
}
__device__ __forceinline__ void red_keep2(float2* p, float x0, float y0, float x1, float y1) {
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(p), "f"(x0), "f"(y0), "f"(x1), "f"(y1), "l"(l2_evict_last())
                 : "memory");
}

// launch `kern` on stream s, with programmatic serialization when pdl is set
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                 cudaStream_t s, bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// mask words covering a plane of `plane` elements (1 bit per 4 nodes)
__host__ __device__ inline int64_t mask_words(int64_t plane) { return (plane + 127) / 128 + 1; }

// coefficient tables and the calling thread's error text (lbib_last_error(NULL))
void fill_coefs_public(const lbib_params& p, Coefs<double>* k);
void fill_coefs_public(const lbib_params& p, Coefs<float>* k);
// the parameter checks of lbib_create (LBIB_OK or LBIB_E_PARAM with the reason)
int check_params_public(const lbib_params* p, std::string* why);
int set_thread_error(int code, const std::string& msg);

// launchers (return cudaError_t of the launch)
// pdl: launch with programmatic serialization (the previous kernel of the
// stream must be the other kernel of the coupled step); nodes_per_thread:
// FP16 storage may update two or four adjacent nodes per thread (1: one; 0:
// the default, two)
// whether the population loads of a lattice should go evict-first in L2:
// both population buffers within 1.5 times the L2 of the current device
bool lattice_l2_first(int precision, int n_species, int64_t plane);

cudaError_t launch_lattice(int precision, int n_species, int bc_y, int forcing,
                           const LatticeArgs& a, const void* coefs, dim3 block,
                           cudaStream_t s, bool pdl = false, int nodes_per_thread = 2);
// the same with confined species (a.dom set, n_species >= 1): one node per
// thread, the confinement paths compiled in (launch_lattice calls it)
cudaError_t launch_lattice_confined(int precision, int n_species, int bc_y, int forcing,
                                    const LatticeArgs& a, const void* coefs, dim3 block,
                                    cudaStream_t s, bool pdl);
// maxv_cell: the largest vertex count of a cell (sizes shared memory and the CTA)
cudaError_t launch_ib(int precision, const IBArgs& a, int maxv_cell, cudaStream_t s,
                      bool pdl = false);
cudaError_t launch_areas(const double2* xy, const int32_t* off, int n_cells, double* area,
                         cudaStream_t s);
// junction partners from the current vertex positions (bins cleared, filled, searched)
cudaError_t launch_junction_renew(const JunctionArgs& j, cudaStream_t s);
cudaError_t launch_init_populations(int precision, int n_species, int nx, int ny,
                                    int64_t pitch, int64_t plane, void* f, void* g,
                                    cudaStream_t s);
// the closure codes of every node from the domain labels (pitch layout)
cudaError_t launch_make_ncode(const int32_t* dom, uint16_t* ncode, int nx, int ny, int bc_y,
                              int64_t pitch, cudaStream_t s);
// the species moments (phi, jx, jy per species; compute type) of the stored
// populations g at every node (the moments a run starts from)
cudaError_t launch_species_moments(int precision, int n_species, int nx, int ny, int64_t pitch,
                                   int64_t plane, const void* g, void* mom, const void* coefs,
                                   cudaStream_t s);
cudaError_t launch_set_species(int precision, int n_species, int s_idx, int nx, int ny,
                               int64_t pitch, int64_t plane, const double* phi, void* g,
                               const void* coefs, cudaStream_t s);

}  // namespace lbib

