"""GPU parity of the cell labelling entry point and of the batched steady
morphogen solve, through the C ABI, against the FP64 oracle.

Tolerances: labels bit-exact (same FP64 predicate on both sides); steady
fields in FP32 storage and arithmetic: relative L-infinity 2e-5 after a
fixed number of steps (eps32 = 6e-8 per update accumulated over a few
thousand relaxation steps), converged step counts within four residual checks.
"""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("seed", [1000, 1001, 1002])
def test_labels_match_oracle_steady_tissues(lb, orc, seed):
    P, T = li.steady_tissue(seed)
    idg, srcg = lb.label_cells(P.nx, P.ny, P.bc_y, T)
    idr, srcr = orc.rasterize(P.nx, P.ny, P.bc_y, T.cell_off, T.xy, T.src_flag)
    assert np.array_equal(idg.cpu().numpy(), idr)
    assert np.array_equal(srcg.cpu().numpy(), srcr)


def test_labels_match_oracle_walls_and_big_cells(lb, orc):
    w = li.config2(nx=300, ny=260, n_cells_side=4)
    idg, srcg = lb.label_cells(w.params.nx, w.params.ny, 1, w.tissue)
    idr, srcr = orc.rasterize(w.params.nx, w.params.ny, 1, w.tissue.cell_off, w.tissue.xy,
                              w.tissue.src_flag)
    assert np.array_equal(idg.cpu().numpy(), idr)
    big = li.scaled_config1(260, 100.0, 400, jitter=0.4).tissue   # brute-force path
    idg, _ = lb.label_cells(260, 260, 0, big)
    idr, _ = orc.rasterize(260, 260, 0, big.cell_off, big.xy, big.src_flag)
    assert np.array_equal(idg.cpu().numpy(), idr)


def _batch(seeds, orc):
    import torch
    Ps, srcs = [], []
    for s in seeds:
        P, T = li.steady_tissue(s)
        _, src = orc.rasterize(P.nx, P.ny, P.bc_y, T.cell_off, T.xy, T.src_flag)
        Ps.append(P)
        srcs.append(src)
    src = torch.as_tensor(np.stack(srcs), device="cuda")
    D = np.array([P.D[0] for P in Ps])
    k = np.array([P.decay[0] for P in Ps])
    s = np.array([P.src_rate[0] for P in Ps])
    return Ps, srcs, src, D, k, s


def test_steady_fixed_steps_match_oracle(lb, orc):
    """tol = 0: every tissue runs exactly max_steps updates on both sides."""
    seeds = [1003, 1004, 1005]
    Ps, srcs, src, D, k, s = _batch(seeds, orc)
    n = 640
    phi, steps, resid = lb.steady_solve(src, D, k, s, tol=0.0, max_steps=n)
    phi = phi.cpu().numpy()
    assert (steps == n).all()
    for b, (P, sr) in enumerate(zip(Ps, srcs)):
        ref, nref, rref, _ = orc.steady(P, sr, tol=0.0, max_steps=n)
        assert nref == n
        assert rel(phi[b], ref[0]) < 2e-5
        assert resid[b] == pytest.approx(rref, rel=1e-2)


def test_steady_converges_like_oracle_and_warm_start(lb, orc):
    seeds = [1006, 1007]
    Ps, srcs, src, D, k, s = _batch(seeds, orc)
    phi, steps, resid = lb.steady_solve(src, D, k, s, tol=1e-6, max_steps=100000)
    phi = phi.cpu().numpy()
    assert (resid <= 1e-6).all()
    refs = []
    for b, (P, sr) in enumerate(zip(Ps, srcs)):
        ref, nref, rref, _ = orc.steady(P, sr, tol=1e-6, max_steps=100000)
        refs.append(ref[0])
        # at r = 1e-6 the FP32 rounding of the per-step change (about 6e-8
        # of max phi) is a few percent of the threshold, which can delay the
        # FP32 decision by a few residual checks
        assert abs(int(steps[b]) - nref) <= 64, (steps[b], nref)
        assert rel(phi[b], ref[0]) < 2.0 * 1e-6 / float(k[b])
    # warm start from the converged field: the populations start at the rest
    # equilibrium w_q phi*, which lacks the non-equilibrium (flux) part of the
    # steady populations, so a short transient remains -- but far shorter
    # than the cold relaxation, and it ends on the same field
    import torch
    phi0 = torch.as_tensor(np.stack(refs).astype(np.float32), device="cuda")
    phi_w, steps_w, resid_w = lb.steady_solve(src, D, k, s, phi0=phi0, tol=1e-6,
                                              max_steps=100000)
    assert (resid_w <= 1e-6).all()
    assert (steps_w < steps // 2).all(), (steps_w, steps)
    # a residual r <= 1e-6 leaves each run within about r / decay of the exact
    # steady field; runs that approach it from different sides can differ by
    # twice that
    bound = 2.0 * 1e-6 / float(min(k))
    assert rel(phi_w.cpu().numpy(), np.stack(refs)) < bound


def test_warm_start_falls_back_on_a_nonfinite_prediction(lb, orc):
    """A prediction holding NaN or inf is abandoned for the cold start at the
    first residual check (16 steps) and then relaxes exactly like a cold run
    started 16 steps later; a sound prediction is kept."""
    import torch
    Ps, srcs, src, D, k, s = _batch([1008, 1009, 1010], orc)
    cold, steps_c, resid_c = lb.steady_solve(src, D, k, s, tol=1e-6, max_steps=100000)
    phi0 = cold.clone()
    phi0[1] = float("nan")
    phi0[2, 5:9, 5:9] = float("inf")
    warm, steps_w, resid_w, fb = lb.steady_solve(src, D, k, s, phi0=phi0, tol=1e-6,
                                                 max_steps=100000, with_fallback=True)
    assert list(fb) == [0, 1, 1]
    assert (resid_w <= 1e-6).all()
    assert steps_w[0] < steps_c[0] // 2
    for b in (1, 2):
        assert steps_w[b] == steps_c[b] + 16
        assert torch.equal(warm[b], cold[b])
    _, _, _, fb_cold = lb.steady_solve(src, D, k, s, tol=1e-6, max_steps=100000,
                                       with_fallback=True)
    assert not fb_cold.any()


def test_cold_and_warm_within_residual_bound_of_converged_field(lb, orc):
    """The true error at r <= tol: a contraction whose slowest mode decays by
    (1 - decay) per step ends within r / decay of its fixed point.  Reference:
    the FP64 oracle relaxed to r <= 1e-12."""
    import torch
    P, T = li.steady_tissue(1011, n=64)
    P.decay[0] = 5e-3
    _, src = orc.rasterize(P.nx, P.ny, P.bc_y, T.cell_off, T.xy, T.src_flag)
    ref, nref, rref, _ = orc.steady(P, src, tol=1e-12, max_steps=200000)
    assert rref <= 1e-12
    dsrc = torch.as_tensor(src[None], device="cuda")
    args = ([P.D[0]], [P.decay[0]], [P.src_rate[0]])
    cold, _, rc = lb.steady_solve(dsrc, *args, tol=1e-6, max_steps=200000)
    warm, _, rw = lb.steady_solve(dsrc, *args, phi0=0.5 * cold, tol=1e-6, max_steps=200000)
    bound = 1e-6 / P.decay[0] + 2e-5   # plus the FP32 rounding floor
    assert rel(cold[0].cpu().numpy(), ref[0]) < bound
    assert rel(warm[0].cpu().numpy(), ref[0]) < bound


def test_steady_uniform_source_closed_form(lb):
    """All nodes are sources: the steady field is src_rate / decay.  From
    zero the uniform field approaches it as 1 - (1 - decay)^n, so a run that
    stops at a per-step relative change r is short of it by r / decay; in
    FP32 the change of one step is resolved to phi's last place (2^-23
    relative), so the stop comes at r <= tol + 2^-23 and the field is within
    (tol + 2^-23) / decay of src_rate / decay."""
    import torch
    src = torch.ones((2, 32, 40), dtype=torch.uint8, device="cuda")
    decay, rate, tol = [1e-2, 5e-3], [1e-3, 2e-3], 1e-7
    phi, steps, resid = lb.steady_solve(src, [0.1, 0.2], decay, rate, tol=tol, max_steps=20000)
    phi = phi.cpu().numpy()
    for s in range(2):
        bound = (tol + 2.0 ** -23) / decay[s]
        assert np.abs(phi[s] / (rate[s] / decay[s]) - 1).max() < bound, s
    assert (steps % 16 == 0).all()


def test_steady_rejects_bad_arguments(lb):
    import torch
    src = torch.ones((1, 16, 16), dtype=torch.uint8, device="cuda")
    with pytest.raises(lb.LbibError) as e:
        lb.steady_solve(src, [0.0], [1e-2], [1e-3])
    assert e.value.code == lb.LBIB_E_PARAM
