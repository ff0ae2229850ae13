"""The build targets sm_103a only and its host code is portable: the GPU
runs on an Arm host, so the host C++ may use no x86 intrinsics or inline
assembly and the build no -march=native (inline PTX in device code is
fine)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2010_06807_gb300", "csrc")


def test_build_targets_sm103a_without_native_flags():
    src = open(os.path.join(ROOT, "paper_2010_06807_gb300", "build.py")).read()
    assert '"arch=compute_103a,code=sm_103a"' in src
    assert "march" not in src and "mtune" not in src


def test_host_sources_have_no_x86_specifics():
    bad = re.compile(r"immintrin|xmmintrin|emmintrin|x86intrin|__asm__|\basm\s*\(|__builtin_ia32")
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cpp", ".h")):
            text = open(os.path.join(CSRC, f)).read()
            assert not bad.search(text), f
    # device code may carry inline PTX, but never x86 headers
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            assert not re.search(r"immintrin|xmmintrin|emmintrin|x86intrin", open(os.path.join(CSRC, f)).read()), f
