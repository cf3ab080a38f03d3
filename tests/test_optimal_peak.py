"""The optimal-peak scoring of the schedulers (experiments optimal): its
enumeration of contraction orders and its optimum (native plan replay of
every order) against the oracle's enumerator and memory model on small
synthetic DAGs -- the same number of orders and the same smallest peak --
and every scheduler's peak at or above that optimum."""
import pytest

import synth
from oracle import dag as D
from oracle import memory as M
from oracle.enumerate import topological_orders

L = pytest.importorskip("paper_2511_02257_b300")
import experiments as E  # noqa: E402


@pytest.mark.parametrize("name,kw,seed", [
    ("multi_meson", dict(n_functions=1, nvec=4, lt=2, prefix_pool=2), 5),
    ("multi_meson", dict(n_functions=2, nvec=4, lt=2, prefix_pool=2), 0),
    ("multi_meson", dict(n_functions=2, nvec=4, lt=2, prefix_pool=2), 41),
    ("baryon", dict(n_functions=1, nvec=3, lt=2), 7),
    ("tiny", dict(n_functions=1), 2)])
def test_optimal_peak_matches_oracle_enumeration(name, kw, seed):
    wl = synth.make_workload(name, seed=seed, **kw)
    nd, _ = L.build_dag(wl, with_data=False)
    od, _ = D.build_from_workload(wl)
    assert 2 <= len(od.non_leaf()) <= 10
    orders = list(topological_orders(od))
    want = min(M.peak_paper(od, o) for o in orders)
    got, count = E.optimal_peak(nd)
    assert (got, count) == (want, len(orders))
    assert sorted(map(tuple, E.contraction_orders(nd))) == sorted(map(tuple, orders))
    for pol in ("naive", "rsgs", "sibling", "tree", "node"):
        assert nd.schedule(pol, "lru", 0)["peak_paper"] >= want
