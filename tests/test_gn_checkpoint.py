"""Host side of the GN-level checkpoint (no GPU): the .npz file written by
GNCheckpoint.save holds the iterate, the iteration index (the random-number
state of the sketches), |g_0|_inf, the held preconditioner's factors, the
counters and the per-iteration record, and load() gives them back unchanged."""
import numpy as np
import pytest


def _cp(with_precond):
    import paper_2401_15758_gb300 as g
    rng = np.random.default_rng(4)
    n, l = 37, 5
    V = rng.standard_normal((n, l)) if with_precond else None
    lam = np.sort(rng.random(l))[::-1] * 10 if with_precond else None
    rec = [{"J": 12.5 + 1e-13, "g_inf": 0.1, "pcg_its": 4, "relres": 3e-7, "sketched": True, "rank": l,
            "kappa_re": 0.0, "alpha": 1.0, "ls_evals": 0, "ls_status": 0},
           {"J": 1.0 / 3.0, "g_inf": 1e-3, "pcg_its": 3, "relres": 8e-7, "sketched": False, "rank": l,
            "kappa_re": 1.0000000001, "alpha": 0.75, "ls_evals": 2, "ls_status": 0}]
    counters = {"fwd": 3, "tlm_online": 40, "adj_online": 41, "tlm_offline": 16, "adj_offline": 16,
                "tlm_kappa": 1, "adj_kappa": 1, "qr_shifted": 0}
    return g.GNCheckpoint(rng.standard_normal(n), 2, 0.123456789012345, 0 if with_precond else -1, V, lam,
                          counters, rec)


@pytest.mark.parametrize("with_precond", [True, False])
def test_checkpoint_round_trip(tmp_path, with_precond):
    import paper_2401_15758_gb300 as g
    cp = _cp(with_precond)
    path = tmp_path / "cp.npz"
    cp.save(path)
    back = g.GNCheckpoint.load(path)
    assert np.array_equal(back.v, cp.v)
    assert (back.next_iter, back.g0_inf, back.sketch_iter) == (cp.next_iter, cp.g0_inf, cp.sketch_iter)
    if with_precond:
        assert np.array_equal(back.V, cp.V) and np.array_equal(back.lam, cp.lam)
    else:
        assert back.V is None and back.lam is None
    assert back.counters == cp.counters
    assert back.record == cp.record   # floats survive bit for bit


def test_checkpoint_format_is_checked(tmp_path):
    import paper_2401_15758_gb300 as g
    path = tmp_path / "cp.npz"
    _cp(True).save(path)
    with np.load(path) as z:
        fields = dict(z)
    fields["format"] = np.int64(g.GNCheckpoint.FORMAT + 1)
    np.savez(path, **fields)
    with pytest.raises(ValueError):
        g.GNCheckpoint.load(path)
