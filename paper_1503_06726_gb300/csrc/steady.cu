// steady.cu -- cell labelling as its own entry point, and the batched steady
// morphogen solve: the D2Q5 relaxation of Sec. 6.1 with u = 0 on a static
// tissue, iterated until the residual r = max|phi^{n+1} - phi^n| /
// max|phi^{n+1}| (checked every `check_every` steps) reaches `tol`.
//
// B tissues of the same lattice size run side by side (grid.z = tissue).
// Each tissue stops on its own: the residual kernel writes phi of the state
// it checked to the output, and the decision kernel freezes a converged
// tissue (its update kernels return at once from then on), so every tissue
// ends on exactly the step count at which it converged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lbib_internal.cuh"

namespace lbib {

// ---------------------------------------------------------------- labels
__global__ void labels_to_ids(uint32_t* packed, uint8_t* src, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t v = packed[i];
    if (src) src[i] = (v == kOutside) ? 0 : (uint8_t)(v & 0xFu);
    packed[i] = (v == kOutside) ? 0u : (v >> 4) + 1u;
}

// ---------------------------------------------------------------- steady D2Q5
struct SteadyArgs {
    const float* gsrc;
    float* gdst;
    const uint8_t* src;   // batch * N source flags (bit 0)
    const float* omegaD;  // per tissue 1/tau_D
    const float* decay;   // per tissue
    const float* srate;   // per tissue
    const int* active;    // per tissue
    float* phi_prev;      // batch * N: phi^{n} stored by flagged updates
    int nx, ny;
    int64_t pitch, plane, tstride;  // tstride: elements per tissue (5 planes)
    int store_prev;
};

// one D2Q5 update of every active tissue: pull, phi, reaction, BGK with u = 0
__global__ void __launch_bounds__(256) steady_update(SteadyArgs a) {
    const int b = blockIdx.z;
    if (!a.active[b]) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const int xm = (x == 0) ? a.nx - 1 : x - 1;
    const int xp = (x == a.nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? a.ny - 1 : y - 1;
    const int yp = (y == a.ny - 1) ? 0 : y + 1;
    const int64_t P = a.plane;
    const float* G = a.gsrc + (int64_t)b * a.tstride;
    const int64_t r0 = (int64_t)y * a.pitch, node = r0 + x;
    float g[5];
    g[0] = __ldg(G + node);
    g[1] = __ldg(G + 1 * P + r0 + xm);
    g[2] = __ldg(G + 2 * P + (int64_t)ym * a.pitch + x);
    g[3] = __ldg(G + 3 * P + r0 + xp);
    g[4] = __ldg(G + 4 * P + (int64_t)yp * a.pitch + x);
    const uint8_t s = a.src[(int64_t)b * a.nx * a.ny + (int64_t)y * a.nx + x];
    const float phi = ((g[0] + g[1]) + (g[2] + g[3])) + g[4];
    const float R = ((s & 1u) ? a.srate[b] : 0.f) - a.decay[b] * phi;
    const float om = a.omegaD[b];
    float* O = a.gdst + (int64_t)b * a.tstride;
    // weights that sum to one exactly in FP32 (1 - 4 w1 is exact): the
    // update creates no mass from their rounding
    constexpr float w1 = (float)(1.0 / 6.0);
    constexpr float w0 = 1.0f - 4.0f * w1;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const float w = q == 0 ? w0 : w1;
        O[q * P + node] = g[q] + om * (phi * w - g[q]) + w * R;
    }
    if (a.store_prev) a.phi_prev[(int64_t)b * a.nx * a.ny + (int64_t)y * a.nx + x] = phi;
}

// phi of the current state, residual against the stored previous phi
__global__ void __launch_bounds__(256) steady_residual(const float* G0, int64_t pitch,
                                                       int64_t plane, int64_t tstride, int nx,
                                                       int ny, const int* active,
                                                       const float* phi_prev, float* phi_out,
                                                       unsigned* dmax, unsigned* pmax) {
    const int b = blockIdx.z;
    if (!active[b]) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    float d = 0.f, pm = 0.f;
    if (x < nx) {
        const int xm = (x == 0) ? nx - 1 : x - 1;
        const int xp = (x == nx - 1) ? 0 : x + 1;
        const int ym = (y == 0) ? ny - 1 : y - 1;
        const int yp = (y == ny - 1) ? 0 : y + 1;
        const float* G = G0 + (int64_t)b * tstride;
        const int64_t r0 = (int64_t)y * pitch;
        const float phi = ((G[r0 + x] + G[plane + r0 + xm]) +
                           (G[2 * plane + (int64_t)ym * pitch + x] + G[3 * plane + r0 + xp])) +
                          G[4 * plane + (int64_t)yp * pitch + x];
        const int64_t o = (int64_t)b * nx * ny + (int64_t)y * nx + x;
        d = fabsf(phi - phi_prev[o]);
        pm = fabsf(phi);
        // a non-finite value counts as +inf (fmaxf would drop a NaN), so the
        // tissue's residual becomes inf / inf = NaN and never passes the test
        if (!isfinite(d)) d = INFINITY;
        if (!isfinite(pm)) pm = INFINITY;
        phi_out[o] = phi;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) {
        d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, k));
        pm = fmaxf(pm, __shfl_xor_sync(0xffffffffu, pm, k));
    }
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) {
        atomicMax(dmax + b, __float_as_uint(d));
        atomicMax(pmax + b, __float_as_uint(pm));
    }
}

// Warm-start fallback: a tissue started from a prediction goes back to the
// cold start (g = 0) when its residual is not finite, or when after this many
// checks it is not below the residual of its first check (the prediction has
// not brought the relaxation closer); its step count runs on.
constexpr int kFallbackChecks = 64;

struct SteadyState {
    int* active;
    int* warm;        // still watched: on the warm start, fewer than kFallbackChecks checks
    int* grow;        // checks so far (warm only)
    int* fellback;    // the warm start was abandoned
    int* reset;       // restart from g = 0 after this check
    float* prevr;     // residual of the first check
};

// per tissue: r = dmax / pmax; freeze converged tissues, reset the maxima,
// abandon failing warm starts
__global__ void steady_decide(int batch, int64_t n, double tol, SteadyState S, unsigned* dmax,
                              unsigned* pmax, long long* steps, double* resid, int* n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    S.reset[b] = 0;
    if (!S.active[b]) return;
    const float d = __uint_as_float(dmax[b]), p = __uint_as_float(pmax[b]);
    const double r = p > 0.f ? (double)d / (double)p : (d > 0.f ? INFINITY : 0.0);
    resid[b] = r;
    steps[b] = n;
    dmax[b] = 0u;
    pmax[b] = 0u;
    if (S.warm[b]) {
        const bool finite = isfinite(r);
        const int c = ++S.grow[b];
        if (c == 1) S.prevr[b] = (float)r;
        if (!finite || (c >= kFallbackChecks && !(r < (double)S.prevr[b]))) {
            S.warm[b] = 0;
            S.fellback[b] = 1;
            S.reset[b] = 1;
            resid[b] = INFINITY;
            return;
        }
        if (c >= kFallbackChecks) S.warm[b] = 0;  // the prediction has helped: stop watching
    }
    if (r <= tol) {
        S.active[b] = 0;
        atomicSub(n_active, 1);
    }
}

// the cold start for the tissues that abandoned their warm start
__global__ void steady_reset(int nx, int64_t pitch, int64_t plane, int64_t tstride,
                             const int* reset, float* g) {
    const int b = blockIdx.z;
    if (!reset[b]) return;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    float* G = g + (int64_t)b * tstride;
    for (int q = 0; q < 5; ++q) G[q * plane + (int64_t)y * pitch + x] = 0.f;
}

__global__ void steady_init(int batch, int nx, int ny, int64_t pitch, int64_t plane,
                            int64_t tstride, const float* phi0, float* g) {
    const int b = blockIdx.z;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const float v = phi0 ? phi0[(int64_t)b * nx * ny + (int64_t)y * nx + x] : 0.f;
    float* G = g + (int64_t)b * tstride;
    constexpr float w1 = (float)(1.0 / 6.0);
    constexpr float w0 = 1.0f - 4.0f * w1;
    for (int q = 0; q < 5; ++q) G[q * plane + (int64_t)y * pitch + x] = (q == 0 ? w0 : w1) * v;
}

struct SteadyLayout {
    int64_t pitch, plane, tstride;
    uint64_t g[2], phi_prev, coef, active, dmax, pmax, steps, resid, nact, total;
    uint64_t warm, grow, fellback, reset, prevr;
};

static SteadyLayout steady_layout(int nx, int ny, int batch) {
    SteadyLayout L;
    L.pitch = (nx + 31) / 32 * 32;
    L.plane = L.pitch * ny;
    L.tstride = 5 * L.plane;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) {
        uint64_t at = o;
        o = (o + bytes + 255) / 256 * 256;
        return at;
    };
    const uint64_t B = (uint64_t)batch, N = (uint64_t)nx * ny;
    L.g[0] = take(B * L.tstride * 4);
    L.g[1] = take(B * L.tstride * 4);
    L.phi_prev = take(B * N * 4);
    L.coef = take(B * 3 * 4);
    L.active = take(B * 4);
    L.dmax = take(B * 4);
    L.pmax = take(B * 4);
    L.steps = take(B * 8);
    L.resid = take(B * 8);
    L.nact = take(4);
    L.warm = take(B * 4);
    L.grow = take(B * 4);
    L.fellback = take(B * 4);
    L.reset = take(B * 4);
    L.prevr = take(B * 4);
    L.total = o;
    return L;
}

}  // namespace lbib

using namespace lbib;

extern "C" {

int lbib_label_cells(int32_t nx, int32_t ny, int32_t bc_y, int32_t n_cells,
                     const int32_t* d_cell_off, const double* d_xy, const uint8_t* d_src_flag,
                     int32_t* d_id, uint8_t* d_src, void* cuda_stream) {
    NvtxRange nvtx_range("lbib_label_cells");
    if (nx < 8 || ny < 8 || bc_y < 0 || bc_y > 1 || n_cells < 0 || !d_id)
        return set_thread_error(LBIB_E_PARAM, "lbib_label_cells: invalid arguments");
    if (n_cells > 0 && (!d_cell_off || !d_xy || !d_src_flag))
        return set_thread_error(LBIB_E_PARAM, "lbib_label_cells: missing cell arrays");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t N = (int64_t)nx * ny;
    cudaError_t e = cudaMemsetAsync(d_id, 0xFF, N * 4, st);
    if (e == cudaSuccess && n_cells > 0) {
        IBArgs a;
        std::memset(&a, 0, sizeof(a));
        a.xy = const_cast<double2*>(reinterpret_cast<const double2*>(d_xy));
        a.off = d_cell_off;
        a.srcf = d_src_flag;
        a.id = reinterpret_cast<uint32_t*>(d_id);
        a.nx = nx;
        a.ny = ny;
        a.bc_y = bc_y;
        a.n_cells = n_cells;
        a.pitch = nx;
        a.plane = (int64_t)nx * ny;
        a.do_move = 0;
        a.do_prep = 1;
        a.do_mask = 1;
        a.do_force = 0;
        // packed labels (cell << 4 | bits, the lower cell index wins) ...
        a.do_ids = 1;
        e = launch_ib(LBIB_FP32, a, kMaxVertsPerCell, st);
        // ... then every containing cell ORs its source bits into the low bits
        if (e == cudaSuccess) {
            a.do_ids = 0;
            a.id = nullptr;
            a.src = d_id;
            a.src_words = 1;
            e = launch_ib(LBIB_FP32, a, kMaxVertsPerCell, st);
        }
    }
    if (e == cudaSuccess) {
        labels_to_ids<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
            reinterpret_cast<uint32_t*>(d_id), d_src, N);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return set_thread_error(LBIB_E_CUDA, std::string("lbib_label_cells: ") +
                                                 cudaGetErrorString(e));
    return LBIB_OK;
}

int lbib_steady_workspace_size(int32_t nx, int32_t ny, int32_t batch, uint64_t* bytes_out) {
    if (nx < 8 || ny < 8 || batch < 1 || batch > 65535 || !bytes_out)
        return set_thread_error(LBIB_E_PARAM, "lbib_steady_workspace_size: invalid arguments");
    *bytes_out = steady_layout(nx, ny, batch).total;
    return LBIB_OK;
}

int lbib_steady_solve(int32_t nx, int32_t ny, int32_t batch, const uint8_t* d_src,
                      const double* D, const double* decay, const double* src_rate,
                      const float* d_phi0, double tol, int64_t max_steps, int32_t check_every,
                      float* d_phi_out, int64_t* steps_out, double* resid_out,
                      int32_t* fallback_out, void* d_workspace, uint64_t ws_bytes,
                      void* cuda_stream) {
    NvtxRange nvtx_range("lbib_steady_solve");
    if (nx < 8 || ny < 8 || batch < 1 || batch > 65535 || !d_src || !D || !decay ||
        !src_rate || !d_phi_out || !steps_out || !resid_out || check_every < 1 ||
        max_steps < 0 || !(tol >= 0.0))
        return set_thread_error(LBIB_E_PARAM, "lbib_steady_solve: invalid arguments");
    const SteadyLayout L = steady_layout(nx, ny, batch);
    if (!d_workspace || ws_bytes < L.total ||
        reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return set_thread_error(LBIB_E_WORKSPACE, "lbib_steady_solve: workspace too small or misaligned");
    std::vector<float> coef((size_t)3 * batch);
    for (int b = 0; b < batch; ++b) {
        if (!(D[b] > 0.0) || !(decay[b] >= 0.0))
            return set_thread_error(LBIB_E_PARAM, "lbib_steady_solve: need D > 0, decay >= 0");
        coef[b] = (float)(1.0 / (3.0 * D[b] + 0.5));
        coef[batch + b] = (float)decay[b];
        coef[2 * batch + b] = (float)src_rate[b];
    }
    char* ws = static_cast<char*>(d_workspace);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float* g[2] = {reinterpret_cast<float*>(ws + L.g[0]), reinterpret_cast<float*>(ws + L.g[1])};
    float* cf = reinterpret_cast<float*>(ws + L.coef);
    int* active = reinterpret_cast<int*>(ws + L.active);
    unsigned* dmax = reinterpret_cast<unsigned*>(ws + L.dmax);
    unsigned* pmax = reinterpret_cast<unsigned*>(ws + L.pmax);
    long long* steps = reinterpret_cast<long long*>(ws + L.steps);
    double* resid = reinterpret_cast<double*>(ws + L.resid);
    int* nact = reinterpret_cast<int*>(ws + L.nact);
    SteadyState S;
    S.active = active;
    S.warm = reinterpret_cast<int*>(ws + L.warm);
    S.grow = reinterpret_cast<int*>(ws + L.grow);
    S.fellback = reinterpret_cast<int*>(ws + L.fellback);
    S.reset = reinterpret_cast<int*>(ws + L.reset);
    S.prevr = reinterpret_cast<float*>(ws + L.prevr);
    std::vector<int> ones((size_t)batch, 1);
    std::vector<double> infs((size_t)batch, INFINITY);
    cudaError_t e = cudaMemcpyAsync(cf, coef.data(), coef.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(active, ones.data(), (size_t)batch * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(resid, infs.data(), (size_t)batch * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(steps, 0, (size_t)batch * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, (size_t)batch * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pmax, 0, (size_t)batch * 4, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nact, &batch, 4, cudaMemcpyHostToDevice, st);
    // a warm start is watched for the fallback; a cold start is not
    if (e == cudaSuccess && d_phi0)
        e = cudaMemcpyAsync(S.warm, ones.data(), (size_t)batch * 4, cudaMemcpyHostToDevice, st);
    else if (e == cudaSuccess)
        e = cudaMemsetAsync(S.warm, 0, (size_t)batch * 4, st);
    for (int* z : {S.grow, S.fellback, S.reset})
        if (e == cudaSuccess) e = cudaMemsetAsync(z, 0, (size_t)batch * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.prevr, 0, (size_t)batch * 4, st);
    const dim3 blk(128), grd((nx + 127) / 128, ny, batch);
    if (e == cudaSuccess) {
        steady_init<<<grd, blk, 0, st>>>(batch, nx, ny, L.pitch, L.plane, L.tstride, d_phi0, g[0]);
        e = cudaGetLastError();
    }
    SteadyArgs a;
    a.src = d_src;
    a.omegaD = cf;
    a.decay = cf + batch;
    a.srate = cf + 2 * batch;
    a.active = active;
    a.phi_prev = reinterpret_cast<float*>(ws + L.phi_prev);
    a.nx = nx;
    a.ny = ny;
    a.pitch = L.pitch;
    a.plane = L.plane;
    a.tstride = L.tstride;
    int cur = 0;
    int64_t n = 0;
    const int64_t host_every = (int64_t)check_every * 8;
    while (e == cudaSuccess && n < max_steps) {
        const int64_t chunk_end = std::min(max_steps, n + host_every);
        for (; n < chunk_end && e == cudaSuccess;) {
            a.gsrc = g[cur];
            a.gdst = g[1 - cur];
            a.store_prev = ((n + 1) % check_every) == 0;
            steady_update<<<grd, blk, 0, st>>>(a);
            e = cudaGetLastError();
            cur = 1 - cur;
            ++n;
            if (e == cudaSuccess && n % check_every == 0) {
                steady_residual<<<grd, blk, 0, st>>>(g[cur], L.pitch, L.plane, L.tstride, nx,
                                                     ny, active, a.phi_prev, d_phi_out, dmax,
                                                     pmax);
                e = cudaGetLastError();
                if (e == cudaSuccess) {
                    steady_decide<<<(batch + 127) / 128, 128, 0, st>>>(
                        batch, n, tol, S, dmax, pmax, steps, resid, nact);
                    e = cudaGetLastError();
                }
                if (e == cudaSuccess && d_phi0) {
                    steady_reset<<<grd, blk, 0, st>>>(nx, L.pitch, L.plane, L.tstride, S.reset,
                                                      g[cur]);
                    e = cudaGetLastError();
                }
            }
        }
        int left = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&left, nact, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && left == 0) break;
    }
    // tissues that ran out of steps: phi of their final state (residual of the
    // last check is kept); the residual kernel also writes phi_out
    if (e == cudaSuccess && n % check_every != 0) {
        // the last partial chunk left phi_prev stale: recompute phi only
        steady_residual<<<grd, blk, 0, st>>>(g[cur], L.pitch, L.plane, L.tstride, nx, ny, active,
                                             a.phi_prev, d_phi_out, dmax, pmax);
        e = cudaGetLastError();
    }
    std::vector<long long> hs((size_t)batch);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.data(), steps, (size_t)batch * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(resid_out, resid, (size_t)batch * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && fallback_out)
        e = cudaMemcpyAsync(fallback_out, S.fellback, (size_t)batch * 4, cudaMemcpyDeviceToHost,
                            st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return set_thread_error(LBIB_E_CUDA, std::string("lbib_steady_solve: ") +
                                                 cudaGetErrorString(e));
    std::vector<int> act((size_t)batch);
    e = cudaMemcpy(act.data(), active, (size_t)batch * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return set_thread_error(LBIB_E_CUDA, std::string("lbib_steady_solve: ") +
                                                 cudaGetErrorString(e));
    for (int b = 0; b < batch; ++b) steps_out[b] = act[b] ? n : hs[b];
    return LBIB_OK;
}

}  // extern "C"
