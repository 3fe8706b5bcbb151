"""The C-ABI library builds, loads and exports every symbol the headers
declare (CPU only: no compute call is made)."""
import ctypes
import os
import re

from paper_2401_14117_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = binding.header_symbols()
    assert "posit_rgemm" in names and len(names) >= 4
    for name in names:
        assert hasattr(lib, name), name
        assert name in binding._SIGS, f"binding lacks {name}"


def test_header_declares_everything_the_binding_marshals():
    names = set(binding.header_symbols())
    assert set(binding._SIGS) <= names


def test_every_header_function_cites_or_explains():
    """Each declaration sits under a comment block (its contract)."""
    for h in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", h)).read()
        for m in re.finditer(r"POSIT_API\s+\w+\s+(posit_\w+)", src):
            before = src[: m.start()].rstrip()
            assert before.endswith("*/"), m.group(1)


def test_product_code_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2401_14117_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "posit_oracle" not in text, f


def test_autotune_argument_errors_need_no_device():
    """posit_autotune rejects bad arguments before any CUDA call."""
    plan = binding.posit_plan(256, 1, 48 * 1024, 0)
    cases = [((0, None, None, 1, 1, [plan]), -1), ((1, None, None, 1, 1, [plan]), -2),
             ((1, 16, None, -1, 1, [plan]), -4), ((1, 16, None, 1, -1, [plan]), -5)]
    for args, code in cases:
        try:
            binding.posit_autotune(*args, reps=1, stream=0)
        except binding.PositError as e:
            assert e.code == code, (args, e.code)
        else:
            raise AssertionError(f"{args} accepted")
    try:
        binding.posit_autotune(1, 16, None, 1, 1, [plan], reps=0, stream=0)
    except binding.PositError as e:
        assert e.code == -8
    else:
        raise AssertionError("reps = 0 accepted")
