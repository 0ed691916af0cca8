"""GPU parity across launch layouts: a seeded sweep of small random jobs run
with the default (occupancy-scored) launch shape, against the oracle.

The default shape depends on the lattice and on the trajectory count, so small
jobs take one team per CTA with slice steps that are odd or do not divide L_t,
narrow slices take several warps per trajectory, and larger counts keep warp
teams.  Every job must give the oracle's W_int and final spins bit for bit,
and the shape the library reports must be a valid one."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="no CUDA device")]

import paper_2304_03311_gb300 as jz  # noqa: E402
from paper_2304_03311_gb300 import build as jzbuild  # noqa: E402


def _jobs(n=36, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(rng.integers(2, 4))
        L = int(2 * rng.integers(1, 33 if d == 2 else 7))
        L_t = int(2 * rng.integers(1, 17))
        l = int(rng.integers(0, L))
        n_traj = int(rng.choice([1, 2, 3, 5, 17, 40, 70]))
        n_step = int(rng.integers(1, 6))
        out.append(dict(d=d, L=L, L_t=L_t, l=l, n_traj=n_traj, n_step=n_step,
                        n_sweep=int(rng.integers(1, 3)), n_therm=int(rng.integers(0, 4)),
                        beta=float(rng.uniform(0.1, 0.6)), seed=int(rng.integers(0, 2**63)),
                        direction=int(rng.choice([1, -1])), traj0=int(rng.integers(0, 1000))))
    return out


JOBS = _jobs()


@pytest.fixture(scope="module")
def ctx():
    jzbuild.build()
    c = jz.ising_replica_init(0, 0, None)
    yield c
    jz.ising_replica_free(c)


@pytest.mark.parametrize("j", JOBS, ids=lambda j: "d{d}L{L}Lt{L_t}n{n_traj}".format(**j))
def test_default_shape_is_bit_exact(ctx, j):
    p = jz.make_params(j["d"], j["L"], j["L_t"], j["beta"], j["l"], j["n_step"], j["n_sweep"],
                       j["n_traj"], j["seed"], n_therm=j["n_therm"], direction=j["direction"],
                       traj0=j["traj0"])
    sh = jz.ising_launch_shape(ctx, p)
    col = ((j["L"] // 2 + 7) // 8) * (j["L"] if j["d"] == 3 else 1)
    assert 1 <= sh["team_threads"] <= sh["cta_threads"] <= 512
    assert sh["team_threads"] % col == 0 and sh["team_threads"] // col >= 1
    if sh["warp"]:
        assert sh["cta_threads"] % 32 == 0 and sh["team_threads"] <= 32
    else:
        assert sh["teams"] == 1 and sh["team_threads"] >= min(32, col * j["L_t"])
    V = 2 * j["L_t"] * j["L"] ** (j["d"] - 1)
    w = torch.empty(j["n_traj"], dtype=torch.int64, device="cuda")
    s = torch.empty(j["n_traj"] * V, dtype=torch.int8, device="cuda")
    jz.jarzynski_run_ex(ctx, p, w, s)
    jz.ising_sync(ctx)
    Wo, So = oracle.run(j["d"], j["L"], j["L_t"], j["beta"], j["l"], j["n_step"], j["n_sweep"],
                        j["n_traj"], j["seed"], n_therm=j["n_therm"], direction=j["direction"],
                        traj0=j["traj0"], want_spins=True)
    np.testing.assert_array_equal(w.cpu().numpy(), Wo)
    np.testing.assert_array_equal(s.cpu().numpy().reshape(j["n_traj"], -1),
                                  So.reshape(j["n_traj"], -1))


def test_the_sweep_reaches_both_layouts(ctx):
    """The random jobs exercise warp teams and one-team CTAs."""
    kinds = set()
    for j in JOBS:
        p = jz.make_params(j["d"], j["L"], j["L_t"], 0.3, j["l"], 2, 1, j["n_traj"], 0)
        kinds.add(jz.ising_launch_shape(ctx, p)["warp"])
    assert kinds == {True, False}


@pytest.mark.parametrize("ts", [3, 5, 7, 10])
def test_odd_and_non_dividing_slice_steps_are_bit_exact(ts):
    """One team per CTA of col * TS threads with TS odd or not dividing L_t
    (3D L = 18: 36 words per slice, L_t = 10), both directions."""
    c = jz.ising_replica_init(0, 0, None)
    try:
        jz.ising_set_threads(c, 3, 18, 10, 36 * ts)
        for dirn in (1, -1):
            p = jz.make_params(3, 18, 10, 0.22, 7, 3, 1, 3, 99, n_therm=2, direction=dirn)
            assert jz.ising_launch_shape(c, p)["team_threads"] == 36 * ts
            w = torch.empty(3, dtype=torch.int64, device="cuda")
            s = torch.empty(3 * 2 * 10 * 18 * 18, dtype=torch.int8, device="cuda")
            jz.jarzynski_run_ex(c, p, w, s)
            jz.ising_sync(c)
            Wo, So = oracle.run(3, 18, 10, 0.22, 7, 3, 1, 3, 99, n_therm=2, direction=dirn,
                                want_spins=True)
            np.testing.assert_array_equal(w.cpu().numpy(), Wo)
            np.testing.assert_array_equal(s.cpu().numpy().reshape(3, -1), So.reshape(3, -1))
    finally:
        jz.ising_replica_free(c)
