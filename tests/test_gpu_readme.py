"""The README's Python examples run as written, and what they print holds:
the quickstart's CG converges, and the batched example solves every system.
The examples are read from README.md (its ```python blocks) so that the
documentation cannot drift from the API."""
import os
import re

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

README = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "README.md")


def _blocks():
    with open(README) as f:
        text = f.read()
    return re.findall(r"```python\n(.*?)```", text, flags=re.S)


def test_readme_has_two_python_examples():
    assert len(_blocks()) == 2


def test_quickstart_runs_and_converges(gk):
    env = {}
    exec(compile(_blocks()[0], "README quickstart", "exec"), env)
    st, A, x0, b = env["st"], env["A"], env["x0"], env["b"]
    assert st.stop_reason == gk.STOP_CONVERGED and st.rel_res_true <= 1.5e-10
    # the solution reproduces the right-hand side
    r = b.clone()
    gk.apply_adv(-1.0, A, x0, 1.0, r)
    assert float(r.norm()) <= 1.5e-10 * float(b.norm())


def test_batched_example_solves_every_system(gk):
    import torch

    import workloads as W
    env = {"W": W, "torch": torch, "gk": gk, "np": np,
           "t": lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()}
    src = _blocks()[1].replace("W.batch_varcoef2d(10_000)", "W.batch_varcoef2d(300)")
    exec(compile(src, "README batched example", "exec"), env)
    res = env["res"]
    assert (res["stop_reason"] == gk.STOP_CONVERGED).all()
    assert (res["rel_res"] <= 1e-10).all()
