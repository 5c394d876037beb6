"""CPU checks of the C ABI: the library builds, loads, and exports every
symbol include/cms.h declares; host-only calls behave.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1108_1320_gb300 import build as b
    b.build()
    from paper_1108_1320_gb300 import cms
    return cms.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "cms.h")).read()
    return sorted(set(re.findall(r"CMS_API\s+[\w\s\*]+?\b(cms_\w+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = _declared()
    for must in ("cms_make_hashes", "cms_sketch_product", "cms_decode", "cms_decode_dense",
                 "cms_sketch_product_plain_f64", "cms_workspace_size", "cms_check_async"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1108_1320_gb300 import cms
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in cms.SIGNATURES, f"binding lacks {name}"


def test_binding_declares_nothing_extra():
    from paper_1108_1320_gb300 import cms
    assert set(cms.SIGNATURES) == set(_declared())


def test_status_strings(lib):
    from paper_1108_1320_gb300 import cms
    for code, name in cms.STATUS.items():
        assert cms.status_string(code) == name


def test_null_arguments_are_rejected_without_cuda(lib):
    # argument checks run before any CUDA call
    assert lib.cms_make_hashes(1, 10, 16, 1, None) == 1
    out = ctypes.c_void_p()
    assert lib.cms_make_hashes(1, 0, 16, 1, ctypes.byref(out)) == 1
    assert lib.cms_make_hashes(1, 10, 16, 0, ctypes.byref(out)) == 1
    assert lib.cms_make_hashes(1, 10, 16, 65, ctypes.byref(out)) == 1
    assert b"d must be" in lib.cms_last_error()
    assert lib.cms_workspace_size(None, 1, 1, 1, 0, None) == 1
    assert lib.cms_decode(None, None, None, 0, None, None) == 1
    assert lib.cms_merge(None, -1, 1, 1, None, None) == 1


def test_build_flags_target_sm103a():
    from paper_1108_1320_gb300 import build as b
    assert "arch=compute_103a,code=sm_103a" in b.ARCH


def test_binding_buffer_checks_without_cuda():
    # the binding's check of caller buffers is plain Python: host tensors,
    # wrong dtypes, non-contiguous views and short buffers are refused
    # before any library call
    import torch
    from paper_1108_1320_gb300 import cms
    with pytest.raises(TypeError):
        cms._check_buf([1.0], "c", "cuda:0")
    with pytest.raises(ValueError, match="CUDA"):
        cms._check_buf(torch.zeros(8), "c", "cuda:0", torch.float32, 8)
    meta = torch.empty((4, 8), device="meta")
    with pytest.raises(ValueError, match="CUDA"):
        cms._check_buf(meta, "c", "cuda:0")


def test_package_exports_every_public_binding_function():
    # every public function and class of the binding is reachable from the
    # package itself (tests and users call paper_1108_1320_gb300.<name>)
    import inspect

    import paper_1108_1320_gb300 as pkg
    from paper_1108_1320_gb300 import cms
    public = [n for n, v in vars(cms).items()
              if not n.startswith("_") and (inspect.isfunction(v) or inspect.isclass(v))
              and getattr(v, "__module__", "") == cms.__name__]
    assert public
    missing = [n for n in public if not hasattr(pkg, n)]
    assert not missing, f"not exported from the package: {missing}"
    assert set(public) <= set(pkg.__all__)


def test_every_package_attribute_the_tests_call_exists():
    # scan the GPU test files for cms.<name> calls made on the package
    # fixture and check each name resolves on the package
    import glob

    import paper_1108_1320_gb300 as pkg
    names = set()
    for path in glob.glob(os.path.join(ROOT, "tests", "test_*.py")):
        src = open(path).read()
        if path.endswith("test_abi.py") or "import paper_1108_1320_gb300 as m\n" not in src:
            continue
        names |= set(re.findall(r"\bcms\.([A-Za-z]\w+)\b", src))
    from paper_1108_1320_gb300 import cms as binding
    missing = [n for n in sorted(names) if not hasattr(pkg, n) and not hasattr(binding, n)]
    assert not missing, missing
    missing_pkg = [n for n in sorted(names) if not hasattr(pkg, n) and not n.startswith("_")]
    assert not missing_pkg, f"tests call these on the package, which lacks them: {missing_pkg}"


def test_noalloc_rejects_n2_beyond_32_bits_without_cuda(lib):
    # the allocation-free entry point refuses the same shapes as the
    # workspace one, with the same text, before any CUDA call: n2 >= 2^31
    # (inner indices are 32-bit in the kernels) is checked before the hashes
    for fn, extra in ((lib.cms_sketch_product_noalloc, (None,)),
                      (lib.cms_sketch_product, (None, 0, None))):
        assert fn(None, 1, None, 1, 1, 1 << 31, 1, 0, None, None, *extra) == 1
        assert b"n2 too large" in lib.cms_last_error()
        assert fn(None, 1, None, 1, 1, -1, 1, 0, None, None, *extra) == 1
        assert b"negative dimension" in lib.cms_last_error()
