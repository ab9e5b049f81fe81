"""The C-ABI library loads and exports every entry point include/svgp.h
declares; ctypes structure layouts match the C compiler's.  No GPU calls."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "svgp.h")


def _declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(svgp_[A-Za-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_00697_gb300 import _lib, build

    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2604_00697_gb300 import _lib

    assert sorted(_lib.EXPORTED) == _declared_functions()
    for n in _lib.EXPORTED:
        assert callable(getattr(_lib, n))


def test_struct_layouts_match_c(tmp_path):
    from paper_2604_00697_gb300 import _lib

    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "svgp.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %d\\n", sizeof(svgp_config), sizeof(svgp_params),'
                   ' sizeof(svgp_batch), sizeof(svgp_grads), offsetof(svgp_batch, N), SVGP_NTERMS);return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(_lib.svgp_config)
    assert int(out[1]) == ctypes.sizeof(_lib.svgp_params)
    assert int(out[2]) == ctypes.sizeof(_lib.svgp_batch)
    assert int(out[3]) == ctypes.sizeof(_lib.svgp_grads)
    assert int(out[4]) == _lib.svgp_batch.N.offset
    assert int(out[5]) == _lib.SVGP_NTERMS


def test_status_strings_without_gpu(lib):
    lib.svgp_status_string.restype = ctypes.c_char_p
    assert lib.svgp_status_string(0) == b"ok"
    assert lib.svgp_status_string(1) == b"invalid argument"


def test_gauss_hermite_rule_matches_numpy(lib):
    """The library's host-side Gauss-Hermite rule (probit likelihood) against
    numpy's hermgauss, and its argument checks.  Host code only."""
    import numpy as np

    from paper_2604_00697_gb300 import _lib

    for n in (1, 2, 3, 7, 20, 32, 64):
        t, w = _lib.svgp_gauss_hermite(n)
        tr, wr = np.polynomial.hermite.hermgauss(n)
        np.testing.assert_allclose(t, tr, rtol=0, atol=1e-12)
        np.testing.assert_allclose(w, wr, rtol=1e-11, atol=1e-300)
    for bad in (0, 65, -3):
        with pytest.raises(_lib.SvgpError):
            _lib.svgp_gauss_hermite(bad)


def test_create_checks_the_precision_before_touching_a_device():
    """svgp_create validates its configuration on the host: an unknown
    precision is an invalid argument; a tensor-core precision (BF16, BF16X3,
    BF16X3K) on a machine without a GB300 is unsupported, not a CUDA error."""
    from paper_2604_00697_gb300 import _lib

    with pytest.raises(_lib.SvgpError) as e:
        _lib.svgp_create(64, 2, 16, prec=4)
    assert e.value.status == _lib.SVGP_ERR_INVALID_ARG
    if _lib.svgp_has_tensor_cores():
        pytest.skip("a tensor-core device is present: the handle would be created")
    for prec in (_lib.SVGP_BF16, _lib.SVGP_BF16X3, _lib.SVGP_BF16X3K):
        with pytest.raises(_lib.SvgpError) as e:
            _lib.svgp_create(64, 2, 16, prec=prec)
        assert e.value.status == _lib.SVGP_ERR_UNSUPPORTED
