"""exa_obj_noalloc: the objective without any allocated scratch.

Some callers cannot allocate device memory (their memory belongs to another allocator, or they run
where cudaMalloc is not allowed).  For them the library keeps the objective's per-CTA partial sums
in a fixed static device array instead of a buffer made by exa_create.  These tests call that entry
point through the C ABI twice in a row and check each result against exa_obj on the same inputs
(the same kernels over the same tiles: equal bit for bit) and against the CPU oracle, and check
that a model needing more partial sums than the array holds is refused with f left untouched.
The file is collected last and passes both alone and after the other tests.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_obj_noalloc_matches_obj_twice():
    from paper_2608_16265_gb300 import binding
    for wl, point in ((synth.acopf(500, 700, 100, seed=1), synth.acopf_point),
                      (synth.rosenbrock(1000), synth.rosenbrock_point)):
        m = binding.exa_create(wl.flat)
        o = oracle.Oracle(wl.flat)
        for seed in (0, 1):  # two calls in a row, different inputs
            x, _, _ = point(wl, seed)
            xt = torch.as_tensor(x, device="cuda")
            f_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
            f_new = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            m.exa_obj(xt, f_ref)
            m.exa_obj_noalloc(xt, f_new)
            torch.cuda.synchronize()
            a, b = float(f_new.item()), float(f_ref.item())
            assert np.float64(a).tobytes() == np.float64(b).tobytes(), (a, b)
            fo = o.obj(x)
            assert abs(a - fo) <= 1e-12 * max(abs(fo), 1e-300), (a, fo)
        m.destroy()


def test_obj_noalloc_refuses_beyond_the_array():
    """65537 objective tiles (one more than the array's 65536 partials) at 32 threads per CTA:
    EXA_E_UNSUPPORTED, and the output keeps its value."""
    from paper_2608_16265_gb300 import binding as B
    from paper_2608_16265_gb300.ir import Model
    n = 65537 * 32
    mod = Model()
    xv = mod.add_var(n)
    mod.add_obj(lambda d: xv[d.k] ** 2, n=n)
    m = B.exa_create(mod.flat(), block=32, flags=B.EXA_FLAG_NO_TUNE)
    assert m.stat("eval_block") == 32
    xt = torch.ones(n, dtype=torch.float64, device="cuda")
    f = torch.full((1,), -3.5, dtype=torch.float64, device="cuda")
    with pytest.raises(B.ExaError) as e:
        m.exa_obj_noalloc(xt, f)
    assert e.value.status == B.EXA_E_UNSUPPORTED and "65537" in str(e.value)
    torch.cuda.synchronize()
    assert float(f.item()) == -3.5
    m.exa_obj(xt, f)  # the allocating call serves the same model
    torch.cuda.synchronize()
    assert float(f.item()) == float(n)
    m.destroy()
