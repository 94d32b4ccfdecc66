"""The C ABI without a GPU: the library builds and loads, exports every function
include/mlt.h declares, its structs match the ctypes mirrors byte for byte, and
its host-only arithmetic (Chebyshev coefficients) agrees with the oracle."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mlt.h")


@pytest.fixture(scope="module")
def L():
    from paper_2103_10516_gb300 import build, mlt
    build.build()
    return mlt


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlt_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 10
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, out, flags=re.M), n


def test_struct_layout_matches_ctypes(L, tmp_path):
    import ctypes
    src = tmp_path / "layout.c"
    structs = [("mlt_mlmc_params", L.mlt_mlmc_params), ("mlt_mlmc_result", L.mlt_mlmc_result),
               ("mlt_learned_params", L.mlt_learned_params), ("mlt_kernel_stat", L.mlt_kernel_stat),
               ("mlt_moments_job", L.mlt_moments_job)]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "mlt.h"', 'int main(void){']
    expect = []
    for cname, cls in structs:
        body.append('printf("%%zu\\n", sizeof(%s));' % cname)
        expect.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            body.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
            expect.append(getattr(cls, f).offset)
    body += ['return 0;}']
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals == expect


def test_constants_match_header(L):
    txt = open(HEADER).read()
    def val(name):
        return int(re.search(r"#define %s\s+\(?(-?\d+)u?\)?" % name, txt).group(1))
    assert val("MLT_EINVAL") == L.MLT_EINVAL and val("MLT_ERANGE") == L.MLT_ERANGE
    assert val("MLT_MAX_LEVELS") == L.MLT_MAX_LEVELS and val("MLT_MAX_DEGREE") == L.MLT_MAX_DEGREE
    assert val("MLT_GRAM") == L.MLT_GRAM and val("MLT_DEVICE_PTRS") == L.MLT_DEVICE_PTRS
    assert val("MLT_REORDER") == L.MLT_REORDER and val("MLT_TRI_CV_CHEB") == L.MLT_TRI_CV["cheb"]
    assert val("MLT_FN_SQRT") == L.MLT_FN["sqrt"] and val("MLT_PREC_FP32") == L.MLT_PREC["fp32"]
    assert val("MLT_NET_NPARAMS") == L.MLT_NET_NPARAMS and val("MLT_NET_HID") == L.MLT_NET_HID


@pytest.mark.parametrize("fn,a,b,n", [("log", 0.1, 8.1, 128), ("sqrt", 0.0, 50.0, 512),
                                       ("exp", -10.0, 10.0, 128), ("inv", 0.5, 3.0, 40),
                                       ("cube", -1.0, 1.0, 9), ("pow", 0.2, 4.0, 64)])
def test_cheb_coeffs_match_oracle(L, O, fn, a, b, n):
    # host-only arithmetic of the library (no device work)
    got = L.mlt_cheb_coeffs(fn, a, b, n, p=1.5)
    ref = O.cheb_coeffs(fn, a, b, n, p=1.5)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.sum(np.abs(ref))


def test_cheb_coeffs_rejects_bad_input(L):
    for args in (("log", -1.0, 2.0, 8), ("log", 1.0, 1.0, 8), ("inv", -1.0, 1.0, 8),
                 ("exp", 0.0, 1.0, 0), ("exp", 0.0, 1.0, 5000)):
        with pytest.raises(L.MLTError) as e:
            L.mlt_cheb_coeffs(*args)
        assert e.value.code == L.MLT_EINVAL


def test_noalloc_binding_rejects_bad_tensors(L):
    """mlt_moments_noalloc hands raw device pointers to the library, which cannot
    see a wrong dtype or a short array: the binding must refuse them first.  With
    host tensors every dtype and length check still runs (they come before the
    device check), so each rejection is exercised without a GPU."""
    import torch
    d, nnz = 4, 6
    good = dict(rowptr=torch.tensor([0, 2, 3, 5, 6], dtype=torch.int64),
                col=torch.tensor([1, 2, 0, 0, 3, 2], dtype=torch.int32),
                vals=torch.ones(nnz, dtype=torch.float64),
                mu=torch.zeros((2, 5), dtype=torch.float64))
    deg = [4, 2]
    bad_cases = [
        ("rowptr", torch.tensor([0, 2, 3, 5, 6], dtype=torch.int32), "int64"),
        ("rowptr", torch.tensor([0, 2, 3, 6], dtype=torch.int64), "entries"),
        ("col", torch.tensor([1, 2, 0, 0, 3, 2], dtype=torch.int64), "int32"),
        ("col", torch.tensor([1, 2, 0], dtype=torch.int32), "at least"),
        ("vals", torch.ones(nnz, dtype=torch.float32), "float64"),
        ("vals", torch.ones(3, dtype=torch.float64), "at least"),
        ("mu", torch.zeros((2, 5), dtype=torch.float32), "float64"),
        ("mu", torch.zeros((1, 5), dtype=torch.float64), "rows"),
        ("mu", torch.zeros((2, 4), dtype=torch.float64), "columns"),
        ("mu", torch.zeros((5, 2), dtype=torch.float64).t(), "contiguous"),
        ("col", [1, 2, 0, 0, 3, 2], "torch tensor"),
    ]
    for name, val, msg in bad_cases:
        args = dict(good)
        args[name] = val
        with pytest.raises(ValueError, match=msg):
            L.mlt_moments_noalloc(d, nnz, args["rowptr"], args["col"], args["vals"], 1.0, -1.0, 1.0, 0, 0,
                                  deg, args["mu"])
    # every check passed but the tensors are host memory: refused as well
    with pytest.raises(ValueError, match="CUDA memory"):
        L.mlt_moments_noalloc(d, nnz, good["rowptr"], good["col"], good["vals"], 1.0, -1.0, 1.0, 0, 0,
                              deg, good["mu"])
