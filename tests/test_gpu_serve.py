"""Continuous-batching server (paper_1512_01977_gb300.serve): every request's
result is the same whether it ran alone or in the mix; a failing request is
retired with its error without disturbing the others; the footprint budget
bounds what is resident."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_01977_gb300 import build, lbm, serve

    build.build()
    lbm.lib()
    return lbm, serve


def _requests():
    # small grids and step counts; staggered arrivals so requests join and leave mid-flight
    specs = [("droplet", "cs", 64, 48, 300, 0.85), ("wave", "vdw", 96, 32, 500, 0.8),
             ("droplet", "vdw", 80, 40, 200, 0.85), ("wave", "cs", 48, 64, 400, 0.9),
             ("droplet", "cs", 120, 60, 350, 0.88), ("wave", "cs", 40, 32, 150, 0.7),
             ("droplet", "cs", 64, 40, 250, 0.5)]
    reqs = [dict(id=i, t_arrive=0.002 * i, kind=k, eos=e, nz=nz, nr=nr, steps=st, T_over_Tc=T)
            for i, (k, e, nz, nr, st, T) in enumerate(specs)]
    reqs[-1]["tau"] = 0.55  # ratio 725 at tau 0.55: expected to go unphysical
    return reqs


def test_served_results_equal_alone(env):
    lbm, serve = env
    reqs = _requests()
    res, stats = serve.serve(reqs, keep_rho=True, max_tick_steps=64)
    assert stats["requests"] == len(reqs)
    by_id = {r.id: r for r in res}
    for req in reqs:
        s, fields = serve.make_solver(req)
        serve.start(s, fields)
        try:
            s.step(req["steps"])
            st = lbm.OK
        except lbm.LbmError as e:
            st = e.code
        r = by_id[req["id"]]
        assert r.status == st, (req, r.status, st)
        if st == lbm.OK:
            alone = lbm.lbm_axi_moments(s.h, req["nz"], req["nr"], want=("rho",))["rho"]
            np.testing.assert_array_equal(r.rho, alone)
            assert r.mass_rweighted == s.mass()[0]
        s.close()
    assert by_id[6].status == lbm.ERR_UNPHYSICAL
    assert sum(1 for r in res if r.status == lbm.OK) == 6
    assert all(r.latency >= 0 and r.t_done >= r.t_start >= 0 for r in res)


def test_budget_bounds_resident_footprint(env):
    lbm, serve = env
    reqs = [r for r in _requests() if r["id"] != 6]
    fp = [lbm.lbm_axi_footprint(r["nz"], r["nr"], 32) for r in reqs]
    budget = max(fp) + min(fp)  # room for at most two of them at once
    res, stats = serve.serve(reqs, budget_bytes=budget, max_tick_steps=64)
    assert stats["completed"] == len(reqs)
    # with two resident at most, every request finished after at least its predecessor-but-one started
    order = sorted(res, key=lambda r: r.t_start)
    for i in range(2, len(order)):
        assert order[i].t_start >= min(o.t_done for o in order[:i]) - 1e-9


def test_unphysical_initial_state_is_retired_at_admission(env):
    """A request whose initial density has psi^2 = rho/3 - P_k < 0 (a CS
    liquid at twice rho_l) is retired with its error when admitted; the
    others run."""
    lbm, serve = env
    reqs = [r for r in _requests() if r["id"] in (0, 1)]
    bad = dict(reqs[0], id=9, t_arrive=0.0)
    orig = serve.make_solver

    def make(req, precision=32, stream=None):
        s, fields = orig(req, precision, stream)
        if req["id"] == 9:
            fields = (fields[0] * 2.0,) + tuple(fields[1:])  # liquid at 2 rho_l: psi^2 < 0
        return s, fields

    serve.make_solver = make
    try:
        res, stats = serve.serve(reqs + [bad], max_tick_steps=64)
    finally:
        serve.make_solver = orig
    by_id = {r.id: r for r in res}
    assert by_id[9].status == lbm.ERR_UNPHYSICAL
    assert by_id[0].status == lbm.OK and by_id[1].status == lbm.OK
    assert stats["requests"] == 3
