"""Host-side checks of the C-ABI boundary (no GPU needed): the library builds
for sm_103a, loads, and exports every entry point that include/lor.h
declares; the Python binding names the same set; and the product path
refuses to run without CUDA tensors (no CPU fallback)."""
import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lor.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lor_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2210_12253_gb300.build import build
    return build()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ("lor_create", "lor_destroy", "lor_set_coefficient", "lor_build_pattern", "lor_assemble",
                     "lor_apply", "lor_apply_backward", "lor_precond_setup", "lor_precond_apply", "lor_pcg_solve"):
        assert required in names


def test_header_documents_every_entry_point():
    """Each declaration's comment cites the passage that defines the call (or
    says it is plumbing with no passage) and states its error behaviour."""
    src = open(os.path.join(ROOT, "include", "lor.h")).read()
    decl = re.compile(r"/\*((?:(?!\*/).)*?)\*/\s*(?:int|const char\*)\s+(lor_[a-z_0-9]+)\s*\(", re.S)
    documented = {}
    for com, name in decl.findall(src):
        cites = re.search(r"Section|Step|Eq\.|Algorithm|[Pp]lumbing|no passage", com)
        errors = re.search(r"LOR_E|Never fails|Always LOR_OK", com)
        documented[name] = bool(cites and errors)
    assert sorted(documented) == declared_entry_points()
    assert all(documented.values()), [n for n, ok in documented.items() if not ok]


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_entry_points() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2210_12253_gb300.lor import EXPORTED
    assert sorted(EXPORTED) == declared_entry_points()


def test_create_error_without_context_is_reported(libpath):
    """lor_create rejects bad configurations before touching the GPU."""
    from paper_2210_12253_gb300 import lor as B
    L = B.load_library(libpath)
    h = ctypes.c_void_p()
    # the last two: 2^31 DOFs exactly, and 2^22 DOFs per axis, whose product wraps to 0 in int64
    for p, nes in ((0, (2, 2, 2)), (B.LOR_MAX_P + 1, (2, 2, 2)), (3, (0, 0, 0)), (1, (2047, 1023, 1023)),
                   (1, ((1 << 22) - 1,) * 3)):
        cfg = B.lor_config(p, *nes)
        rc = L.lor_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None)
        assert rc == B.LOR_EINVAL
        assert L.lor_last_error(None)
        assert not h.value
    assert L.lor_create(None, None, None, None) == B.LOR_EINVAL
    fake = ctypes.c_void_p(16)  # never dereferenced: the sizes are rejected first
    for p, nel, ndof in ((0, 8, 27), (3, 0, 27), (3, 8, 1 << 31), (3, 1 << 60, 1000)):
        rc = L.lor_create_general(ctypes.byref(h), p, nel, ndof, fake, fake, None, None)
        assert rc == B.LOR_EINVAL and not h.value


def test_device_allocation_failure_is_reported(libpath, monkeypatch):
    """An allocation failure injected on the host (LOR_DEVICE_ALLOC_LIMIT)
    comes back as LOR_ENOMEM with no context, before any device call."""
    from paper_2210_12253_gb300 import lor as B
    L = B.load_library(libpath)
    h = ctypes.c_void_p()
    cfg = B.lor_config(2, 2, 2, 2)
    monkeypatch.setenv("LOR_DEVICE_ALLOC_LIMIT", "64")  # below the 648-byte vertex copy
    rc = L.lor_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(16), None)
    assert rc == B.LOR_ENOMEM and not h.value
    assert b"LOR_DEVICE_ALLOC_LIMIT" in L.lor_last_error(None)


def test_product_path_needs_cuda_tensors(libpath):
    from paper_2210_12253_gb300 import LOR
    with pytest.raises(TypeError):
        LOR(2, 1, 1, 1, torch.zeros(8 * 3, dtype=torch.float64))


def test_binding_constants_match_the_header():
    """Every enumerator and status code the header defines has the same value
    in the binding."""
    import re
    from paper_2210_12253_gb300 import lor as B
    text = open(os.path.join(ROOT, "include", "lor.h")).read()
    pairs = re.findall(r"\b(LOR_[A-Z0-9_]+)\s*=\s*(\d+)", text)
    pairs += re.findall(r"#define\s+(LOR_[A-Z0-9_]+)\s+(\d+)\b", text)
    assert len(pairs) >= 15
    for name, value in pairs:
        assert hasattr(B, name), name
        assert getattr(B, name) == int(value), name


def test_every_entry_point_rejects_a_null_context(libpath):
    """The header's error contract on the host side: every call that takes a
    context returns LOR_EINVAL for a NULL one (before touching the GPU), and
    lor_destroy(NULL) is a no-op."""
    from paper_2210_12253_gb300 import lor as B
    L = B.load_library(libpath)
    skip = {"lor_last_error", "lor_launch_count", "lor_create", "lor_destroy"}
    checked = 0
    for name in B.EXPORTED:
        if name in skip:
            continue
        fn = getattr(L, name)
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint):
                args.append(0)
            elif t is ctypes.c_double:
                args.append(0.0)
            else:
                args.append(None)  # pointers, the context and the stream
        assert fn(*args) == B.LOR_EINVAL, name
        checked += 1
    assert checked >= 20
    assert L.lor_destroy(None) == B.LOR_OK
