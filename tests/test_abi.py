"""Host-side checks of the C ABI: the library loads, exports every declared
entry point, and rejects bad arguments before touching a device."""

import ctypes as C
import os
import re

import pytest

from paper_2609_16478_b300 import ahoc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ahoc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ahoc_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = ahoc.lib()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(ahoc.SYMBOLS)


def test_status_strings():
    L = ahoc.lib()
    for s in range(9):
        assert L.ahoc_status_string(s).startswith(b"AHOC_")
    assert L.ahoc_status_string(99) == b"unknown ahoc_status"


def test_workspace_bytes_and_validation():
    L = ahoc.lib()
    nb2 = ahoc.workspace_bytes(2, [64, 64])
    nb3 = ahoc.workspace_bytes(3, [16, 16, 16])
    assert nb2 > 2 * 64 * 64 * 8 and nb3 > 2 * 16 ** 3 * 8
    # grows with the Krylov cap
    assert ahoc.workspace_bytes(2, [64, 64], restart=200) > nb2
    out = C.c_size_t(0)
    bad = [(4, [64, 64, 64, 64]), (2, [48, 64]), (2, [4, 64]), (3, [8192, 8, 8])]
    for dim, N in bad:
        n = (C.c_int64 * len(N))(*N)
        st = L.ahoc_workspace_bytes(dim, n, None, C.byref(out))
        assert st in (ahoc.AHOC_EINVAL, ahoc.AHOC_EUNSUPPORTED)
        assert L.ahoc_last_error()


def test_plan_create_rejects_before_allocating():
    L = ahoc.lib()
    h = C.c_void_p(0)
    n = (C.c_int64 * 2)(64, 64)
    lo = (C.c_double * 2)(0.0, 0.0)
    hi = (C.c_double * 2)(1.0, 1.0)
    # NULL alpha
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, None, None, None, None) == ahoc.AHOC_EINVAL
    # empty box
    assert L.ahoc_plan_create(C.byref(h), 2, n, hi, hi, C.c_void_p(256), None, None, None) == ahoc.AHOC_EINVAL
    # unsupported precision / preconditioner
    o = ahoc.ahoc_opts()
    o.prec = 7
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), None, C.byref(o), None) == ahoc.AHOC_EUNSUPPORTED
    # misaligned caller workspace
    o = ahoc.ahoc_opts()
    o.workspace = C.c_void_p(8)
    o.workspace_bytes = 1 << 40
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), None, C.byref(o), None) == ahoc.AHOC_EINVAL
    # too-small caller workspace
    o.workspace = C.c_void_p(4096)
    o.workspace_bytes = 16
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), None, C.byref(o), None) == ahoc.AHOC_ENOMEM
    assert h.value is None
    # NULL plan to the compute calls
    assert L.ahoc_matvec(None, None, None) == ahoc.AHOC_EINVAL
    assert L.ahoc_solve(None, None, None, C.c_double(1e-12), None) == ahoc.AHOC_EINVAL
    assert L.ahoc_solve_from(None, None, None, None, C.c_double(1e-12), None) == ahoc.AHOC_EINVAL
    assert L.ahoc_plan_destroy(None) == ahoc.AHOC_OK
    assert L.ahoc_n_gamma(None) == -1


def test_no_unresolved_library_symbols():
    """Every symbol of the library's own namespace is defined (templates instantiated)."""
    import subprocess
    out = subprocess.run(["nm", "-D", "--undefined-only", ahoc.LIB_PATH], capture_output=True, text=True).stdout
    assert "ahoc" not in out, out


def test_every_bdata_field_reaches_each_problem():
    """ahoc_plan_create splits the batch's boundary-data arrays per problem:
    every field of ahoc_bdata must be forwarded (a field missing there is
    silently zero)."""
    import re
    src = open(os.path.join(ROOT, "paper_2609_16478_b300", "csrc", "plan.cu")).read()
    hdr = open(os.path.join(ROOT, "include", "ahoc.h")).read()
    body = hdr[hdr.index("typedef struct {", hdr.index("Boundary data")):hdr.index("} ahoc_bdata;")]
    fields = re.findall(r"const double\* (\w+);", body)
    assert len(fields) >= 6
    create = src[src.index("ahoc_status ahoc_plan_create("):]
    create = create[:create.index("s = plan_load(")]
    for f in fields:
        assert "bb.%s = bd->%s" % (f, f) in create, f


def test_struct_layouts_and_constants_match_header(tmp_path):
    """The binding's ctypes mirrors of ahoc_bdata, ahoc_opts and ahoc_info
    have the header's field offsets and sizes, and its constants the
    header's values: a C program compiled against include/ahoc.h prints
    them (a field missing from the header fails to compile)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("ahoc_bdata", ahoc.ahoc_bdata), ("ahoc_opts", ahoc.ahoc_opts), ("ahoc_info", ahoc.ahoc_info)]
    consts = [n for n in dir(ahoc) if re.fullmatch(r"AHOC_(E[A-Z]+|OK|FP64|MIXED|TUNE_[A-Z_]+)", n)]
    assert {"AHOC_OK", "AHOC_EINTERNAL", "AHOC_MIXED", "AHOC_TUNE_DST_RADIX"} <= set(consts)
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ahoc.h"', "int main(void) {"]
    for sname, cls in structs:
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (sname, sname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s*)0)->%s));'
                         % (sname, fname, sname, fname, sname, fname))
    for n in consts:
        lines.append('  printf("%s %%d\\n", (int)%s);' % (n, n))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = dict(l.split(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for sname, cls in structs:
        assert int(out[sname].split()[1]) == C.sizeof(cls), sname
        for fname, _ in cls._fields_:
            off, size = map(int, out["%s.%s" % (sname, fname)].split())
            desc = getattr(cls, fname)
            assert (off, size) == (desc.offset, desc.size), (sname, fname, off, size, desc.offset, desc.size)
    for n in consts:
        assert int(out[n]) == getattr(ahoc, n), n


def test_misaligned_device_arrays_are_refused_on_the_host():
    """A device array of doubles at an address that is not a multiple of 8
    is refused with AHOC_EINVAL before any launch (an 8-byte load from it
    would fault the kernel)."""
    L = ahoc.lib()
    n = (C.c_int64 * 2)(16, 16)
    lo = (C.c_double * 2)(0.0, 0.0)
    hi = (C.c_double * 2)(1.0, 1.0)
    h = C.c_void_p()
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(260), None, None, None) == ahoc.AHOC_EINVAL
    assert b"aligned" in L.ahoc_last_error()
    bd = ahoc.ahoc_bdata()
    bd.g_N = C.c_void_p(1028)
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), C.byref(bd), None, None) == ahoc.AHOC_EINVAL
    assert b"aligned" in L.ahoc_last_error()
    assert h.value is None
    assert L.ahoc_poisson_noalloc(2, n, lo, hi, C.c_void_p(4100), C.c_void_p(8192), None) == ahoc.AHOC_EINVAL
    assert b"aligned" in L.ahoc_last_error()


def test_indefinite_shift_is_unsupported():
    """beta / alpha < 0 (the high-wavenumber problem's indefinite Helmholtz
    v-equation) is a valid problem outside the library: AHOC_EUNSUPPORTED,
    before any allocation; a non-finite shift is an invalid argument."""
    L = ahoc.lib()
    n = (C.c_int64 * 2)(64, 64)
    lo = (C.c_double * 2)(0.0, 0.0)
    hi = (C.c_double * 2)(1.0, 1.0)
    h = C.c_void_p()
    o = ahoc.ahoc_opts()
    o.shift = -100.0
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), None, C.byref(o), None) == \
        ahoc.AHOC_EUNSUPPORTED
    assert b"indefinite" in L.ahoc_last_error()
    nbytes = C.c_size_t()
    assert L.ahoc_workspace_bytes(2, n, C.byref(o), C.byref(nbytes)) == ahoc.AHOC_EUNSUPPORTED
    o.shift = float("nan")
    assert L.ahoc_plan_create(C.byref(h), 2, n, lo, hi, C.c_void_p(256), None, C.byref(o), None) == ahoc.AHOC_EINVAL
    assert h.value is None
