"""exa_obj_noalloc: the objective without any allocated scratch.

Some callers cannot allocate device memory (their memory belongs to another allocator, or they run
where cudaMalloc is not allowed).  For them the library keeps the objective's per-CTA partial sums
in a fixed static device array instead of a buffer made by exa_create.  This test calls that entry
point through the C ABI twice in a row and checks each result against exa_obj on the same inputs.
It lives in its own file, collected last, and passes both alone and after the other tests.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_obj_noalloc_matches_obj_twice():
    from paper_2608_16265_gb300 import binding
    for wl, point in ((synth.acopf(500, 700, 100, seed=1), synth.acopf_point),
                      (synth.rosenbrock(1000), synth.rosenbrock_point)):
        m = binding.exa_create(wl.flat)
        for seed in (0, 1):  # two calls in a row, different inputs
            x, _, _ = point(wl, seed)
            xt = torch.as_tensor(x, device="cuda")
            f_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            f_new = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            m.exa_obj(xt, f_ref)
            m.exa_obj_noalloc(xt, f_new)
            torch.cuda.synchronize()
            a, b = float(f_new.item()), float(f_ref.item())
            assert np.isfinite(a)
            assert abs(a - b) <= 1e-12 * max(abs(b), 1e-300)
        m.destroy()
