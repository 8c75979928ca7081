"""The allocation-free entry point, lbib_step_noalloc, against lbib_step.

Callers that may not allocate device memory while they run (a framework's
memory pool owns the device, or a plug-in must keep its footprint fixed) use
lbib_step_noalloc with buffers they already own; its intermediate planes live
in a static device array in the library.  These tests give it the same state
as a context, run two calls in a row and compare populations and vertex
positions with the context's lbib_step after each call: FP64 storage at the
FP64 parity tolerance used elsewhere (relative L-infinity 1e-10), FP32
storage at the tolerance of the ensemble-against-single-tissue test (the same
kernels, only the atomic order of the spreading differs: populations 1e-5
relative, positions 1e-9 LU).  The call synchronises its stream, so the
stream is idle when it returns.  The file is collected last and holds its own
state, so it passes alone or after the other tests.
"""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


def _split_state(blob, w, es, plane):
    """Population and vertex sections of an lbib_get_state() blob."""
    S = w.params.n_species
    o = 16
    f = blob[o:o + 9 * plane * es]
    o += 9 * plane * es
    g = blob[o:o + 5 * S * plane * es]
    o += 5 * S * plane * es
    V = w.tissue.n_vertices
    xy = blob[o:o + V * 16].view(np.float64).reshape(V, 2)
    return f, g, xy


def _lattice(raw, n_planes, plane, pitch, nx, ny, dtype=np.float64):
    """The nx*ny nodes of each plane (row and plane padding are never written)."""
    v = raw.view(dtype)
    return np.stack([v[q * plane:q * plane + pitch * ny].reshape(ny, pitch)[:, :nx]
                     for q in range(n_planes)]).astype(np.float64)


def _rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a - b).max())


def _two_calls(precision, tol_pop, tol_xy):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()

    w = li.config1()
    T = w.tissue
    p = w.params
    cp = lbib.make_params(p, precision)
    es = 8 if precision == lbib.LBIB_FP64 else 4
    dt = np.float64 if es == 8 else np.float32
    pitch = (p.nx + 63) // 64 * 64
    plane = pitch * p.ny + 1536 // es

    sim = lbib.Simulation(p, precision, T.n_vertices, T.n_cells)
    sim.set_cells(T)
    f0, g0, xy0 = _split_state(sim.get_state(), w, es, plane)
    assert np.array_equal(xy0, T.xy)

    dev = torch.device("cuda")
    d_f = torch.from_numpy(f0.copy()).to(dev)
    d_g = torch.from_numpy(g0.copy()).to(dev)
    d_xy = torch.from_numpy(T.xy.copy()).to(dev)
    d_off = torch.from_numpy(T.cell_off.astype(np.int32)).to(dev)
    d_L0 = torch.from_numpy(T.rest_len.copy()).to(dev)
    d_k = torch.from_numpy(T.k_spring.copy()).to(dev)
    d_p = torch.from_numpy(T.pressure.copy()).to(dev)
    d_s = torch.from_numpy(T.src_flag.astype(np.uint8)).to(dev)
    cs = torch.cuda.current_stream()
    torch.cuda.synchronize()

    for n in (3, 4):   # two calls in a row, odd then even step counts
        lbib.lbib_step_noalloc(cp, T.n_cells, d_off.data_ptr(), d_xy.data_ptr(),
                               d_L0.data_ptr(), d_k.data_ptr(), d_p.data_ptr(), d_s.data_ptr(),
                               d_f.data_ptr(), d_g.data_ptr(), n, cs.cuda_stream)
        assert cs.query(), "the call returns with its stream idle"
        sim.step(n)
        fr, gr, xyr = _split_state(sim.get_state(), w, es, plane)
        S = p.n_species
        fn = _lattice(d_f.cpu().numpy(), 9, plane, pitch, p.nx, p.ny, dt)
        gn = _lattice(d_g.cpu().numpy(), 5 * S, plane, pitch, p.nx, p.ny, dt)
        assert _rel(fn, _lattice(fr, 9, plane, pitch, p.nx, p.ny, dt)) < tol_pop
        assert _rel(gn, _lattice(gr, 5 * S, plane, pitch, p.nx, p.ny, dt)) < tol_pop
        assert np.abs(fn).max() > 0 and np.abs(gn).max() > 0
        assert np.abs(d_xy.cpu().numpy() - xyr).max() < tol_xy
    sim.close()


def test_noalloc_matches_context_two_calls():
    from paper_1503_06726_gb300 import lbib
    _two_calls(lbib.LBIB_FP64, 1e-10, 1e-12)


def test_noalloc_fp32_matches_context_two_calls():
    from paper_1503_06726_gb300 import lbib
    _two_calls(lbib.LBIB_FP32, 1e-5, 1e-9)


def test_noalloc_rejects_oversized_lattice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import lbib
    w = li.config1()
    w.params.nx = w.params.ny = 512
    cp = lbib.make_params(w.params, lbib.LBIB_FP64)
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(lbib.LbibError) as e:
        lbib.lbib_step_noalloc(cp, 0, 0, 0, 0, 0, 0, 0, dummy.data_ptr(), dummy.data_ptr(), 1,
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.code == lbib.LBIB_E_WORKSPACE
    assert "4 MiB" in lbib.lbib_last_error(None)
