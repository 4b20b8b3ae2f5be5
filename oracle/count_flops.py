"""Count the method's FP64 arithmetic per element-step on the oracle's own source.

TEST INFRASTRUCTURE ONLY: run as a script, it prints the counts that bench.py quotes beside
the kernel's executed count (tests/test_oracle_flop_count.py re-counts and compares).

The oracle's source is evaluated over counting numbers (oracle_ad.cpp): every FP64 addition or
subtraction, multiplication and division of a step is counted, and special functions
(sqrt, sin, cos, atan2, floor, fabs) are counted as calls.  "flops" below is
additions + multiplications + divisions, each one operation (the oracle contracts nothing
into fused multiply-adds); special calls are listed beside it.

Workloads (seeded recipes of rodgen, the same as the benchmark's), each in a general state
(rodgen.perturbed: bent, twisted and spinning elements, so that every element takes the
rotation maps' general branches; a straight rod at rest skips them):
  packing: 300 rods of the packing's recipe (n ~ U{16..256}, gravity) placed without overlap
           in a box of the 10^4-rod packing's density (0.31 m), one step without contact (the
           step kernel's arithmetic) and one with the cell-list contact of the placement (no
           overlap there, so only the broad phase and the candidate tests add work; touching
           pairs add ~100 flops each);
  carpet:  16 x 16 of the carpet's identical 50-element rods (base couple, Stokes drag), one
           step (per element-step the same count as the 64 x 64 carpet).
"""
from __future__ import annotations

import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import rodgen  # noqa: E402
from oracle.oracle import Oracle  # noqa: E402


def per_element_step(problem, dt: float, n_steps: int = 1, contact: bool = None):
    """{class: operations per element-step, "flops": add + mul + div} of n_steps oracle steps."""
    p = problem if contact is None else problem.replace(contact=contact)
    _, counts = Oracle(p).step_count(p.state(), dt, n_steps)
    units = p.n_elems * n_steps
    out = {k: v / units for k, v in counts.items()}
    out["flops"] = (counts["add"] + counts["mul"] + counts["div"]) / units
    out["special"] = sum(counts[k] for k in ("sqrt", "sincos", "atan2", "floor", "fabs")) / units
    return out


def packing_sample():
    return rodgen.perturbed(rodgen.random_packing(n_rods=300, box=0.31, seed=1234), seed=1)


def carpet_sample():
    return rodgen.perturbed(rodgen.cilia_carpet(side=16), seed=1)


def counts():
    pk = packing_sample()
    carpet = carpet_sample()
    return {
        "packing_step_without_contact": per_element_step(pk, 5e-6, contact=False),
        "packing_step_with_contact": per_element_step(pk, 5e-6, contact=True),
        "carpet_step": per_element_step(carpet, 1e-5),
    }


if __name__ == "__main__":
    print(json.dumps(counts(), indent=1))
