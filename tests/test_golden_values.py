"""The oracle and the library against values the paper states
(tests/golden/paper_values.json, each entry with its passage)."""
import json
import os

import numpy as np

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_legendre_nodes():
    g = GOLD["legendre_nodes"]
    # P_1(x) = x: the oracle's degree-1 column is the node itself
    np.testing.assert_array_equal(O.legendre(g["p"], 1)[:, 1], g["x"])


def test_weight_quantile_worked_example():
    g = GOLD["weight_quantile"]
    f = np.asarray(g["flux"], np.float32)
    for q, w in zip(g["quantiles"], g["w"]):
        _, _, got, _ = O.prep(f, np.ones_like(f), np.ones(f.shape, np.uint8), quantile=q)
        assert got == w


def test_default_options_are_the_papers():
    a, s, c = GOLD["adam"], GOLD["stop_rules"], GOLD["clean"]
    o = O.make_opts()
    assert (o.lr, o.beta1, o.beta2, o.eps) == (a["lr"], a["beta1"], a["beta2"], a["eps"])
    assert (o.window, o.tol) == (s["window"], s["tol"])
    assert (o.clean_every, o.clean_max) == (c["every"], c["max_updates"])
    from paper_2512_24840_gb300 import lasp
    g = lasp.default_opts()
    assert np.float32(g.lr) == np.float32(a["lr"]) and np.float32(g.eps) == np.float32(a["eps"])
    assert np.float32(g.beta1) == np.float32(a["beta1"]) and np.float32(g.beta2) == np.float32(a["beta2"])
    assert (g.window, np.float32(g.tol)) == (s["window"], np.float32(s["tol"]))
    assert (g.clean_every, g.clean_max) == (c["every"], c["max_updates"])
