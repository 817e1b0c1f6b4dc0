"""The per-thread ephemeris path at table sizes around the shared Chebyshev
basis's limit: tables of up to 16 coefficients per segment are summed from one
basis per force evaluation (kept in shared memory), longer ones with the basis
made per body.  12 and 16 coefficients take the first form, 17 and 24 the
second; both against the FP64 oracle's textbook recurrence on the same table
(App. A: the planets from a Chebyshev table).

Tolerances as in test_gpu_parity: the table lookup within 1e-14 of the
oracle's sum, positions after 60 days within 1e-9 AU.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_04666_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N_BODIES = 256


@pytest.fixture(scope="module")
def K():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_04666_gb300 import build as B, kete
    B.build()
    k = kete.Kete(0)
    yield k
    k.close()


@pytest.fixture(scope="module")
def bodies():
    seed = W.SEED_BASE
    ps = W.make_planets(seed)
    states, _ = W.population(seed, ps, N_BODIES)
    return ps, states


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("n_coef", [12, 16, 17, 24])
def test_table_size_lookup_and_propagation(K, bodies, n_coef):
    ps, states = bodies
    eph = W.build_ephemeris(ps, W.T0 - 32.0, W.T0 + 96.0, seg_len=16.0, n_coef=n_coef)
    assert eph.n_coef == n_coef
    K.load_ephem(eph.to_bytes())
    orc = O.Oracle(eph.to_bytes())
    # the lookup itself
    rng = np.random.default_rng(n_coef)
    t = rng.uniform(eph.t_start, eph.t_end, 64)
    for body in (0, 3, 5):
        pos, vel = K.ephem_eval(_dev(t), body)
        pos = pos.cpu().numpy(); vel = vel.cpu().numpy()
        for i, ti in enumerate(t):
            _, p, v = orc.ephem(body, ti)
            assert np.abs(pos[i] - p).max() < 1e-14 * max(1, np.abs(p).max())
            assert np.abs(vel[i] - v).max() < 1e-15 * 50
    # one 60-day leg: steps shorter than the leg evaluate the planets per
    # thread (no node rows), through the path the table size selects
    t1 = W.T0 + 60.0
    st = _dev(states.copy())
    ep = _dev(np.full(N_BODIES, W.T0))
    status = K.propagate(st, ep, t1)
    stats = K.get_stats()
    assert stats["force_evals"] > stats["node_evals"]
    ref, _, ref_status, _ = orc.propagate_many(orc.force_model(), states,
                                               np.full(N_BODIES, W.T0), t1)
    assert (status.cpu().numpy() == 0).all() and (ref_status == 0).all()
    err = np.abs(st.cpu().numpy()[:3] - ref[:3]).max()
    assert err < 1e-9, (n_coef, err)
