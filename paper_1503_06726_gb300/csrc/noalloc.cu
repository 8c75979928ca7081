// noalloc.cu -- coupled steps for callers that cannot allocate device memory.
//
// Some callers are not allowed to call cudaMalloc (or any allocator) while
// they run: code inside a framework whose memory pool owns the whole device,
// or plug-ins that must not change the device's memory footprint after
// start-up.  For them this file provides lbib_step_noalloc(), which runs the
// same kernels as lbib_step() on state buffers the caller already owns, and
// keeps every intermediate plane (the second population buffer, the spread
// force, the source bits, the velocity and the diagnostic words) in one
// file-scope static device array of kScratchBytes.  Every GPU that loads the
// library holds that array until the process exits.  The call reads the
// diagnostic words back and synchronises its stream before it returns, so it
// must not be called while that stream is being captured into a graph.
#include <cstring>
#include <mutex>
#include <string>

#include "lbib_internal.cuh"

namespace lbib {

constexpr uint64_t kScratchBytes = 4ull << 20;  // 4 MiB
constexpr int kMaxDevices = 64;

// The scratch planes.  Host code must not pass the symbol itself to a kernel:
// on the host it names a stand-in, not device memory.  The device address is
// looked up once per device with cudaGetSymbolAddress (see scratch_ptr).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
static cudaError_t scratch_ptr(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

static uint64_t up256(uint64_t v) { return (v + 255) / 256 * 256; }

}  // namespace lbib

using namespace lbib;

extern "C" int lbib_step_noalloc(const lbib_params* params, int32_t n_cells,
                                 const int32_t* d_cell_off, double* d_xy,
                                 const double* d_rest_len, const double* d_k_spring,
                                 const double* d_pressure, const uint8_t* d_src_flag, void* d_f,
                                 void* d_g, int32_t n_steps, void* cuda_stream) {
    std::string why;
    if (check_params_public(params, &why) != LBIB_OK)
        return set_thread_error(LBIB_E_PARAM, "lbib_step_noalloc: " + why);
    Layout L;
    if (!make_layout(*params, 0, 0, &L) || n_steps < 0 || n_cells < 0)
        return set_thread_error(LBIB_E_PARAM, "lbib_step_noalloc: invalid parameters");
    if (params->noflux_mask)
        return set_thread_error(LBIB_E_PARAM,
                                "lbib_step_noalloc: confined species need a context's domain plane");
    if (params->junction_period > 0)
        return set_thread_error(LBIB_E_PARAM,
                                "lbib_step_noalloc: cell junctions need a context");
    if (params->mass_sources || params->pressure_nodes || params->node_sources)
        return set_thread_error(LBIB_E_PARAM,
                                "lbib_step_noalloc: mass sources and pressure nodes need a context");
    if (!d_f || (params->n_species > 0 && !d_g) ||
        (n_cells > 0 && (!d_cell_off || !d_xy || !d_rest_len || !d_k_spring || !d_pressure ||
                         !d_src_flag)))
        return set_thread_error(LBIB_E_PARAM, "lbib_step_noalloc: missing buffer");
    // the kernels move populations, positions and constants in vector and
    // word accesses of these sizes
    auto misaligned = [](const void* p, uintptr_t a) {
        return p && reinterpret_cast<uintptr_t>(p) % a != 0;
    };
    if (misaligned(d_f, 16) || misaligned(d_g, 16) || misaligned(d_xy, 16) ||
        misaligned(d_rest_len, 8) || misaligned(d_k_spring, 8) || misaligned(d_pressure, 8) ||
        misaligned(d_cell_off, 4))
        return set_thread_error(LBIB_E_PARAM,
                                "lbib_step_noalloc: d_f, d_g, d_xy need 16-byte alignment, "
                                "d_rest_len, d_k_spring, d_pressure 8 bytes, d_cell_off 4 bytes");
    if (n_steps == 0) return LBIB_OK;

    // scratch plan: second population buffer, force, velocity, source bits, diag
    const uint64_t P = (uint64_t)L.plane;
    const uint64_t o_f2 = 0;
    const uint64_t o_g2 = up256(o_f2 + 9 * P * L.es);
    const uint64_t o_force = up256(o_g2 + (uint64_t)5 * params->n_species * P * L.es);
    const uint64_t o_u = up256(o_force + 2 * P * L.cs);
    const uint64_t o_src = up256(o_u + 2 * P * L.cs);
    const uint64_t o_diag = up256(o_src + P);
    const uint64_t need = up256(o_diag + kDiagWords * 4);
    if (need > kScratchBytes)
        return set_thread_error(LBIB_E_WORKSPACE,
                                "lbib_step_noalloc: lattice needs " + std::to_string(need) +
                                    " scratch bytes, more than the static 4 MiB");

    void* base = nullptr;
    cudaError_t e = scratch_ptr(&base);
    if (e != cudaSuccess)
        return set_thread_error(LBIB_E_CUDA, std::string("lbib_step_noalloc: ") +
                                                 cudaGetErrorString(e));
    char* sc = static_cast<char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    Coefs<double> kd;
    Coefs<float> kf;
    fill_coefs_public(*params, &kd);
    fill_coefs_public(*params, &kf);
    const void* coefs = params->precision == LBIB_FP64 ? (const void*)&kd : (const void*)&kf;

    // the scratch keeps the previous call's contents: reset what must start empty
    e = cudaMemsetAsync(sc + o_force, 0, 2 * P * L.cs, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc + o_src, 0, P, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc + o_diag, 0, kDiagWords * 4, st);

    void* fbuf[2] = {d_f, sc + o_f2};
    void* gbuf[2] = {d_g, sc + o_g2};
    LatticeArgs la;
    std::memset(&la, 0, sizeof(la));
    la.force = sc + o_force;
    la.id = nullptr;  // no output step: only source bits are labelled
    la.src = reinterpret_cast<uint8_t*>(sc + o_src);
    la.u = sc + o_u;
    la.diag = reinterpret_cast<uint32_t*>(sc + o_diag);
    la.nx = params->nx;
    la.ny = params->ny;
    la.pitch = L.pitch;
    la.plane = L.plane;
    la.out = 0;
    la.ib = n_cells > 0 ? 1 : 0;
    la.l2_first = lattice_l2_first(params->precision, params->n_species, L.plane) ? 1 : 0;
    IBArgs ia;
    std::memset(&ia, 0, sizeof(ia));
    ia.xy = reinterpret_cast<double2*>(d_xy);
    ia.L0 = d_rest_len;
    ia.k = d_k_spring;
    ia.off = d_cell_off;
    ia.pres = d_pressure;
    ia.srcf = d_src_flag;
    ia.vforce = nullptr;
    ia.force = sc + o_force;
    ia.id = nullptr;
    ia.src = la.src;
    ia.do_ids = 0;
    ia.u = la.u;
    ia.diag = la.diag;
    ia.nx = params->nx;
    ia.ny = params->ny;
    ia.bc_y = params->bc_y;
    ia.n_cells = n_cells;
    ia.pitch = L.pitch;
    ia.plane = L.plane;
    ia.tension = params->tension;
    ia.do_mask = 1;
    ia.write_vforce = 0;
    ia.do_force = 1;

    int cur = 0;
    if (e == cudaSuccess && n_cells > 0) {
        ia.do_move = 0;
        ia.do_prep = 1;
        e = launch_ib(params->precision, ia, kMaxVertsPerCell, st);
    }
    for (int left = n_steps; left > 0 && e == cudaSuccess; --left) {
        la.fsrc = fbuf[cur];
        la.fdst = fbuf[1 - cur];
        la.gsrc = gbuf[cur];
        la.gdst = gbuf[1 - cur];
        e = launch_lattice(params->precision, params->n_species, params->bc_y, params->forcing,
                           la, coefs, dim3(128, 1, 1), st);
        if (e == cudaSuccess && n_cells > 0) {
            ia.do_move = 1;
            ia.do_prep = left > 1 ? 1 : 0;
            e = launch_ib(params->precision, ia, kMaxVertsPerCell, st);
        }
        cur = 1 - cur;
    }
    // leave the state in the caller's buffers
    if (e == cudaSuccess && cur == 1) {
        e = cudaMemcpyAsync(d_f, fbuf[1], 9 * P * L.es, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && params->n_species > 0)
            e = cudaMemcpyAsync(d_g, gbuf[1], (size_t)5 * params->n_species * P * L.es,
                                cudaMemcpyDeviceToDevice, st);
    }
    uint32_t diag[kDiagCheckAddr + 1] = {0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(diag, sc + o_diag, sizeof(diag), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return set_thread_error(LBIB_E_CUDA, std::string("lbib_step_noalloc: ") +
                                                 cudaGetErrorString(e));
    if (diag[kDiagCheck])
        return set_thread_error(LBIB_E_CHECK,
                                "lbib_step_noalloc: checking build: an access failed its bounds or "
                                "alignment check (site " + std::to_string(diag[kDiagCheckSite]) +
                                    ") and was skipped");
    if (diag[kDiagNonFinite] || diag[kDiagGeometry])
        return set_thread_error(LBIB_E_NONFINITE,
                                "lbib_step_noalloc: a non-finite value or blown-up cell appeared");
    return LBIB_OK;
}
