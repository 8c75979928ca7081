// Host-side state of one tissue (the opaque handle of the C ABI), kept apart
// from the kernel headers: no kernel reads it.
#pragma once

#include <string>

#include "lbib_internal.cuh"

// One tissue (the opaque handle of the C ABI).
struct lbib_ctx {
    lbib_params p;
    int maxV = 0, maxC = 0;
    char* ws = nullptr;
    uint64_t bytes = 0;
    cudaStream_t stream = nullptr;
    lbib::Layout L;
    int cur = 0;           // buffer holding the current post-collision populations
    int nV = 0, nC = 0;
    int maxv_cell = 0;     // largest vertex count of a cell
    bool fields_valid = false;
    bool vforce_valid = false;
    lbib::Coefs<double> kd;
    lbib::Coefs<float> kf;
    dim3 block{128, 1, 1};
    bool mass_ctrl = false;      // target areas set: the area controller is on
    int lattice_npt = 0;  // FP16 storage: nodes per thread (1, 2 or 4; 0 = the default, 2)
    int64_t nstep = 0;          // steps since lbib_set_cells / lbib_set_state (junction renewal)
    bool l2_first = false;      // population loads evict-first (lattice nearly fits in L2)
    bool mom_valid = false;     // the no-flux closure's moments of buffer `cur` are current
    // graph of a two-step chunk, keyed by the buffer parity it starts from
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    // the same two steps whose last IB launch only moves (the end of an
    // lbib_advance call), keyed the same way
    cudaGraphExec_t tail[2] = {nullptr, nullptr};
    int chunk_nC = -1;
    // pinned staging of lbib_set_cell_params (pressure then source flags), and
    // the event of its last upload (the buffer is reused once that is done)
    char* hstage = nullptr;
    cudaEvent_t hstage_done = nullptr;
    bool hstage_pending = false;
    // the asynchronous readback of the cell outputs (lbib_get_cells_async):
    // its copy stream, the events before and after its copies, the pinned
    // diagnostic words read back with it; while one is pending, work that
    // writes the vertex positions or the areas first waits for rb_done
    cudaStream_t rb_stream = nullptr;
    cudaEvent_t rb_ready = nullptr, rb_done = nullptr;
    uint32_t* rb_diag = nullptr;
    bool rb_pending = false;
    std::string err;

    template <typename T>
    T* at(uint64_t off) const { return reinterpret_cast<T*>(ws + off); }
};

namespace lbib {
// order the context stream after a pending asynchronous readback (work that
// writes the vertex positions or the cell areas must not overtake its copies)
inline cudaError_t rb_fence(lbib_ctx* c, cudaStream_t s) {
    return c->rb_pending ? cudaStreamWaitEvent(s, c->rb_done, 0) : cudaSuccess;
}
// kernel arguments of a context (its buffers, parity src_buf)
LatticeArgs ctx_lattice_args(lbib_ctx* c, int src_buf, bool out);
IBArgs ctx_ib_args(lbib_ctx* c, bool move, bool prep, bool out_next);
}  // namespace lbib
