"""The checking build (-DLBIB_CHECK): the kernels test the bounds and the
alignment of every vector, atomic and indexed access of the hot path before
making it, skip an access that fails, and the host reports LBIB_E_CHECK.

  - the coupled step (FP64, FP32, FP16 with two and four nodes per thread; walls;
    junctions; mass sources and pressure nodes), confined species under the
    no-flux closure, the ensemble (both schedules), the allocation-free step and the sums run
    in the checking build without a single failed check;
  - a cell whose offsets claim more vertices than the arrays hold (the
    allocation-free step reads offsets only on the device) is caught by the
    vertex check and reported as LBIB_E_CHECK.  The vertex buffer passed there
    really holds twice the vertices the offsets admit, so the access the check
    stops stays inside memory the test owns in either build.

Each case runs in a child process with LBIB_CHECK=1, which loads the checking
library (the parent may hold the plain one).
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(code: str, timeout: int = 900):
    env = dict(os.environ, LBIB_CHECK="1")
    prog = textwrap.dedent("""
        import sys
        sys.path.insert(0, {root!r})
        import numpy as np
        import torch
        import lbib_inputs as li
        from paper_1503_06726_gb300 import lbib
        L = lbib.load()
        assert lbib._lib is not None
        assert "_build_check" in L._name, L._name
    """).format(root=ROOT) + textwrap.dedent(code)
    r = subprocess.run([sys.executable, "-c", prog], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r.stdout


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def test_check_build_hot_path_clean():
    out = _child("""
        def run(w, prec, n, prep=None):
            p, T = w.params, w.tissue
            sim = lbib.Simulation(p, prec, T.n_vertices, T.n_cells)
            sim.set_cells(T)
            if prep:
                prep(sim)
            sim.step(n)
            f = sim.fields(lbib.LBIB_RHO | lbib.LBIB_U | lbib.LBIB_X | lbib.LBIB_AREA)
            sim.sums()
            sim.advance(3)
            sim.step(1)
            sim.fields(lbib.LBIB_U)
            sim.close()
            return f
        run(li.config1(), lbib.LBIB_FP64, 20)
        for prec in (lbib.LBIB_FP32, lbib.LBIB_FP16):
            run(li.config2(nx=128, ny=128, n_cells_side=2), prec, 9)
        run(li.config3(), lbib.LBIB_FP32, 4)    # 9,801 cells: the 64-thread IB kernel
        run(li.config3(n=512), lbib.LBIB_FP16, 5)   # one species: the staged quad update
        run(li.config2_junctions(), lbib.LBIB_FP32, 12)
        g = li.config2_growth()
        def grow(sim):
            sim.set_mass_sources(g.mass_rate, g.target_area)
            sim.set_pressure_nodes(g.pressure_mask)
        run(g, lbib.LBIB_FP32, 6, grow)
        # confined species under the closure
        t = li.turing(n=256)
        sim = lbib.Simulation(t.params, lbib.LBIB_FP32, 0, 0)
        sim.set_domains(t.domains)
        for s in range(t.params.n_species):
            sim.set_species(s, t.phi0[s])
        sim.step(10)
        sim.fields(lbib.LBIB_PHI)
        sim.close()
        # the ensemble
        ws = li.config4(seed=44, n_tissues=3, n_steps=4, side_min=96, side_max=160)
        ens = lbib.Ensemble([w.params for w in ws], [w.tissue for w in ws])
        ens.step(4)
        ens.status()
        ens.schedule(lbib.LBIB_ENS_SPLIT)
        ens.step(3)
        ens.status()
        for i in range(len(ws)):
            ens.fields(i)
        ens.close()
        print("clean")
    """)
    assert "clean" in out


def test_check_build_catches_bad_cell_offsets():
    out = _child("""
        w = li.config1()
        p, T = w.params, w.tissue
        cp = lbib.make_params(p, lbib.LBIB_FP32)
        es = 4
        pitch = (p.nx + 63) // 64 * 64
        plane = pitch * p.ny + 1536 // es
        dev = torch.device("cuda")
        V = T.n_vertices                      # 64
        d_f = torch.zeros(9 * plane, dtype=torch.float32, device=dev)
        d_g = torch.zeros(5 * p.n_species * plane, dtype=torch.float32, device=dev)
        # vertex arrays of 2V entries; the offsets admit V and the first cell
        # claims V + 36 of them
        xy = np.concatenate([T.xy, T.xy])
        d_xy = torch.from_numpy(xy.copy()).to(dev)
        d_off = torch.tensor([0, V + 36, V], dtype=torch.int32, device=dev)
        d_L0 = torch.from_numpy(np.concatenate([T.rest_len] * 2)).to(dev)
        d_k = torch.from_numpy(np.concatenate([T.k_spring] * 2)).to(dev)
        d_p = torch.zeros(2, dtype=torch.float64, device=dev)
        d_s = torch.zeros(2, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        try:
            lbib.lbib_step_noalloc(cp, 2, d_off.data_ptr(), d_xy.data_ptr(), d_L0.data_ptr(),
                                   d_k.data_ptr(), d_p.data_ptr(), d_s.data_ptr(),
                                   d_f.data_ptr(), d_g.data_ptr(), 2,
                                   torch.cuda.current_stream().cuda_stream)
            print("no error")
        except lbib.LbibError as e:
            print("code", e.code, lbib.lbib_last_error(None))
    """)
    assert "code -8" in out, out
