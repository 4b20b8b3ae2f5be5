"""The method's FP64 work per element-step, counted on the oracle's own source (oracle_ad.cpp
over counting numbers; oracle/count_flops.py), and the figures bench.py quotes beside the
kernel's executed count.

Pins of the counting build: it advances the state bit for bit like the oracle, its counts grow
exactly in proportion to the number of steps and of identical rods, and the benchmark's
constants are the counts of oracle/count_flops.py.
"""
import importlib.util
import os

import numpy as np

import rodgen
from oracle.count_flops import counts, per_element_step
from oracle.oracle import Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_counting_build_advances_the_state_like_the_oracle():
    p = rodgen.perturbed(rodgen.cilia_carpet(side=2, n=12), seed=3)
    o = Oracle(p)
    ref = o.step(*p.state(), dt=1e-5, n_steps=4, t=0.3)
    got, c = o.step_count(p.state(), 1e-5, 4, t=0.3)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert c["add"] > 0 and c["mul"] > 0 and c["div"] > 0


def test_counts_scale_with_steps_and_identical_rods():
    # a free, bent and spinning rod: every step takes the same branches
    one = rodgen.perturbed(rodgen.cantilever(n=20), seed=4).replace(clamp_base=None, tip_force=None)
    _, c1 = Oracle(one).step_count(one.state(), 1e-5, 1)
    _, c3 = Oracle(one).step_count(one.state(), 1e-5, 3)
    assert all(c3[k] == 3 * c1[k] for k in c1), (c1, c3)
    # copies of the rod: the count is affine in the number of copies (a few operations per
    # step, such as the stage times, do not depend on the ensemble)
    x, v, Q, w = one.state()

    def copies(m):
        rep = lambda a: np.concatenate([a] * m, axis=-1)
        q = one.replace(n_elem=rep(one.n_elem), rest_len=rep(one.rest_len), radius=rep(one.radius),
                        youngs=rep(one.youngs), shear_mod=rep(one.shear_mod), density=rep(one.density),
                        x=rep(x), v=rep(v), Q=rep(Q), w=rep(w))
        return Oracle(q).step_count(q.state(), 1e-5, 1)[1]

    c2, c4 = copies(2), copies(4)
    assert all(c4[k] - c1[k] == 3 * (c2[k] - c1[k]) for k in c1), (c1, c2, c4)
    assert all(0 <= c1[k] - (c2[k] - c1[k]) <= 10 for k in c1)


def test_bench_quotes_the_oracle_counts():
    b = _bench()
    got = counts()
    step = got["packing_step_without_contact"]
    assert abs(b.ORACLE_FLOPS_PER_UNIT["pack_one_step"] - step["flops"]) < 0.01
    assert abs(b.ORACLE_SPECIAL_PER_UNIT["pack_one_step"] - step["special"]) < 0.01
    assert abs(b.ORACLE_FLOPS_PER_UNIT["pack_steps"] - got["carpet_step"]["flops"]) < 0.01
    assert abs(b.ORACLE_SPECIAL_PER_UNIT["pack_steps"] - got["carpet_step"]["special"]) < 0.01
    contact = got["packing_step_with_contact"]["flops"] - step["flops"]
    assert abs(b.ORACLE_CONTACT_FLOPS_PER_UNIT - contact) < 0.01
