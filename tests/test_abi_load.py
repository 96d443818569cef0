"""The C-ABI library builds, loads without a GPU, and exports every function include/exa.h
declares; the generated kernels of every workload compile with NVRTC for sm_103a (no device
needed)."""
import os
import re

import pytest

import synth
from tests.helpers import all_ops_model

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="exa.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(exa_[a-z_0-9]+)\s*\(", src)))


def test_exports_match_header():
    from paper_2608_16265_gb300 import binding
    lib = binding.load()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(binding.EXPORTS) == names


def test_every_header_is_exported():
    """Every include/*.h function is exported by libexa.so and listed by the binding."""
    from paper_2608_16265_gb300 import binding
    lib = binding.load()
    headers = sorted(h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h"))
    assert headers == ["exa.h", "exa_probe.h"]
    for n in declared_functions("exa_probe.h"):
        assert hasattr(lib, n), n
    assert sorted(binding.PROBE_EXPORTS) == declared_functions("exa_probe.h")


@pytest.mark.parametrize("name,flat", [
    ("all_ops", lambda: all_ops_model().flat()),
    ("rosenbrock", lambda: synth.rosenbrock(20).flat),
    ("acopf", lambda: synth.acopf(6, 9, 2).flat),
    ("pde", lambda: synth.pde(6).flat),
])
def test_generated_kernels_compile(name, flat):
    from paper_2608_16265_gb300 import binding
    binding.exa_compile_check(flat())


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("upfront", [False, True])
def test_generated_variants_compile(precision, upfront):
    """Every code-generator variant the tuner can pick compiles for sm_103a: both precisions, both
    emission orders, with and without a launch-bounds register cap, both L2 prefetch depths, two
    warp sets per instance, inputs loaded one pattern ahead, inputs staged in shared memory, the
    fused step kernels, on the
    two-stage ACOPF (all pattern kinds, scenario-indexed variables, per-scenario parameters)."""
    from paper_2608_16265_gb300 import binding
    flat = synth.two_stage_acopf(5, 7, 2, 3, seed=1).flat
    flags = binding.EXA_FLAG_UPFRONT if upfront else 0
    binding.exa_compile_check(flat, precision=precision, block=128, flags=flags)
    binding.exa_compile_check(flat, precision=precision, block=64, flags=flags, min_blocks=16)
    for pf in (binding.EXA_FLAG_PF_COLUMNS, binding.EXA_FLAG_PF_GATHERS):  # L2 prefetch variants
        binding.exa_compile_check(flat, precision=precision, block=128, flags=flags | pf)
    binding.exa_compile_check(flat, precision=precision, block=128, flags=flags | binding.EXA_FLAG_LANES2)
    if not upfront:
        binding.exa_compile_check(flat, precision=precision, block=64, min_blocks=12,
                                  flags=flags | binding.EXA_FLAG_LAZY_LOADS)
    binding.exa_compile_check(flat, precision=precision, block=64, min_blocks=14,  # fused step kernels
                              flags=flags | binding.EXA_FLAG_FUSED_STEP)
    for lazy in ((0, binding.EXA_FLAG_LAZY_LOADS) if not upfront else (0,)):  # shared-memory staging
        binding.exa_compile_check(flat, precision=precision, block=128, min_blocks=4,
                                  flags=flags | lazy | binding.EXA_FLAG_STAGE_SMEM)


def test_compile_check_rejects_bad_ir():
    from paper_2608_16265_gb300 import binding, ir
    m = ir.Model()
    x = m.add_var(3)
    m.add_obj(lambda d: x[0] * x[1], n=1)
    fl = m.flat()
    fl.patterns[0].vop[-1] = 99  # unknown opcode
    with pytest.raises(binding.ExaError) as e:
        binding.exa_compile_check(fl)
    assert e.value.status == binding.EXA_E_INVALID
    fl = m.flat()
    fl.patterns[0].va[-1] = fl.patterns[0].vb[-1]  # a node with two parents: not a tree
    with pytest.raises(binding.ExaError) as e:
        binding.exa_compile_check(fl)
    assert "tree" in str(e.value)
