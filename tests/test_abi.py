"""The C-ABI library builds, loads and exports every symbol that
include/accord.h declares; the ctypes structs match the C layout; host-side
argument checks answer without touching a GPU."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "accord.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2412_11554_gb300 import build
    build.build()
    from paper_2412_11554_gb300 import accord
    return accord.load_library()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(accord_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for want in ("accord_fit", "accord_loss", "accord_grad", "accord_workspace_bytes", "accord_default_opts"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (accord_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_export():
    from paper_2412_11554_gb300 import accord
    assert set(accord.EXPORTS) == set(declared_functions())


def test_struct_layout_matches_c():
    """Compile a probe against the header with gcc and compare sizeof/offsetof
    with the ctypes mirrors."""
    from paper_2412_11554_gb300.accord import AccordOpts, AccordPathEntry, AccordStats
    fields = {"accord_opts": AccordOpts, "accord_stats": AccordStats, "accord_path_entry": AccordPathEntry}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for cname, cls in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "probe.c"), os.path.join(d, "probe")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for cname, cls in fields.items():
        assert int(got[cname]) == ctypes.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f


def test_plain_c_program_links_and_calls_the_library(lib):
    """A program built against include/accord.h as C11 (gcc) and as C++17
    (g++) and linked with libaccord.so: defaults, workspace sizing, status
    strings and host-side argument errors, with no device work."""
    src = r"""
#include <stdio.h>
#include <string.h>
#include "accord.h"
int main(void) {
  accord_opts o;
  accord_default_opts(&o);
  if (o.precision != ACCORD_MIXED_BF16X3 || o.max_iter != 500) return 1;
  size_t bf = accord_workspace_bytes(1000, 4000, &o);
  o.precision = ACCORD_MIXED_TF32X3;
  size_t tf = accord_workspace_bytes(1000, 4000, &o);
  o.precision = ACCORD_FP64;
  size_t f64 = accord_workspace_bytes(1000, 4000, &o);
  if (!(bf > 0 && tf > bf && f64 > 0)) return 2;
  if (strlen(accord_status_string(ACCORD_ENOMEM)) == 0) return 3;
  long long nnz = -1;
  if (accord_to_csr(0, (void*)16, &o, (int64_t*)16, NULL, NULL, 0, (int64_t*)&nnz) != ACCORD_EINVAL) return 4;
  if (accord_fit(NULL, 10, 10, 0.1, &o, (void*)16, NULL, 0, NULL) != ACCORD_EINVAL) return 5;
  printf("ok %zu %zu %zu\n", bf, tf, f64);
  return 0;
}
"""
    libdir = os.path.dirname(lib._name)
    # the same program as C11 and as C++17 (the header's extern "C" block)
    for compiler, std, ext in (("gcc", "-std=c11", "c"), ("g++", "-std=c++17", "cpp")):
        with tempfile.TemporaryDirectory() as d:
            c, exe = os.path.join(d, "use." + ext), os.path.join(d, "use")
            open(c, "w").write(src)
            subprocess.run([compiler, std, "-Wall", "-Werror", "-I", os.path.dirname(HEADER), "-o", exe, c,
                            "-L", libdir, "-laccord", f"-Wl,-rpath,{libdir}"], check=True)
            r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.startswith("ok "), (compiler, r.returncode, r.stdout, r.stderr)


def test_defaults_and_workspace_sizing(lib):
    from paper_2412_11554_gb300 import accord
    o = accord.accord_default_opts()
    assert (o.precision, o.max_iter, o.max_backtracks, o.penalize_diag) == (accord.MIXED_BF16X3, 500, 60, 1)
    assert (o.tau0, o.beta, o.kkt_tol, o.lipschitz) == (1.0, 0.5, 1e-8, 0.0)
    small = accord.accord_workspace_bytes(100, 200, precision="fp64")
    big = accord.accord_workspace_bytes(1000, 40000)
    assert 0 < small < big
    # dense Omega and Omega+ alone need 2 * 4 * p^2 bytes in mixed mode
    assert big >= 2 * 4 * 40000 ** 2
    assert accord.accord_workspace_bytes(0, 10) == 0
    assert accord.accord_workspace_bytes(10, 10, beta=1.5) == 0
    # TF32x3 planes take 4 bytes an element instead of 2: the five plane pairs
    # (X, X^T, Y twice, Delta) grow by 2 * 2 * (2 n p + 3 p n + p^2) bytes at
    # most the 1 KB rounding of each sub-buffer
    n, p = 1000, 4000
    bf = accord.accord_workspace_bytes(n, p, precision="bf16x3")
    tf = accord.accord_workspace_bytes(n, p, precision="tf32x3")
    grow = 2 * 2 * (n * p + n * p + 2 * p * n + p * p)
    assert abs((tf - bf) - grow) <= 16 * 1024
    ptf = accord.accord_path_workspace_bytes(200, 300, [np.arange(150), np.arange(200)], 2, precision="tf32x3")
    pbf = accord.accord_path_workspace_bytes(200, 300, [np.arange(150), np.arange(200)], 2, precision="bf16x3")
    assert ptf > pbf > 0


def test_invalid_arguments_rejected_on_host(lib):
    """Argument checks happen before any device call, so they work here."""
    from paper_2412_11554_gb300 import accord
    o = accord.accord_default_opts()
    # sparse export: missing Omega / row_ptr / nnz, p < 1, buffers missing for cap > 0
    nz = ctypes.c_int64(-1)
    dptr = ctypes.c_void_p(16)
    assert lib.accord_to_csr(10, None, ctypes.byref(o), dptr, dptr, dptr, 4, ctypes.byref(nz)) == accord.EINVAL
    assert nz.value == 0
    assert lib.accord_to_csr(10, dptr, ctypes.byref(o), None, dptr, dptr, 4, ctypes.byref(nz)) == accord.EINVAL
    assert lib.accord_to_csr(10, dptr, ctypes.byref(o), dptr, dptr, dptr, 4, None) == accord.EINVAL
    assert lib.accord_to_csr(0, dptr, ctypes.byref(o), dptr, dptr, dptr, 4, ctypes.byref(nz)) == accord.EINVAL
    assert lib.accord_to_csr(10, dptr, ctypes.byref(o), dptr, None, None, 4, ctypes.byref(nz)) == accord.EINVAL
    assert lib.accord_to_csr(1 << 31, dptr, ctypes.byref(o), dptr, dptr, dptr, 4, ctypes.byref(nz)) == accord.EINVAL
    st = accord.AccordStats()
    dummy = ctypes.c_void_p(16)
    assert lib.accord_fit(None, 10, 10, 0.1, ctypes.byref(o), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    assert lib.accord_fit(dummy, 0, 10, 0.1, ctypes.byref(o), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    assert lib.accord_fit(dummy, 10, 10, -1.0, ctypes.byref(o), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    bad = accord.accord_default_opts(beta=0.0)
    assert lib.accord_fit(dummy, 10, 10, 0.1, ctypes.byref(bad), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    bad = accord.accord_default_opts(precision=7)
    assert lib.accord_fit(dummy, 10, 10, 0.1, ctypes.byref(bad), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    assert st.status == accord.EINVAL
    assert lib.accord_fit_f64(dummy, 10, 10, 0.1, ctypes.byref(o), dummy, None, 0, None) == accord.EUNSUPPORTED
    st.status, st.iters = 99, 99                        # a NULL X still fills the stats
    assert lib.accord_fit_f64(None, 10, 10, 0.1, ctypes.byref(o), dummy, None, 0, ctypes.byref(st)) == accord.EINVAL
    assert (st.status, st.iters) == (accord.EINVAL, 0)
    # refit: missing Omega_hat, phi outside [0, 1], negative epBIC gamma
    assert lib.accord_refit(dummy, 10, 10, 0.1, 0.5, None, ctypes.byref(o), dummy, None, 0,
                            ctypes.byref(st)) == accord.EINVAL
    assert lib.accord_refit(dummy, 10, 10, 0.1, 1.5, dummy, ctypes.byref(o), dummy, None, 0,
                            ctypes.byref(st)) == accord.EINVAL
    bad = accord.accord_default_opts(epbic_gamma=-1.0)
    assert lib.accord_refit(dummy, 10, 10, 0.1, 0.5, dummy, ctypes.byref(bad), dummy, None, 0,
                            ctypes.byref(st)) == accord.EINVAL
    # lambda path: argument checks before any device call
    import numpy as np
    rows = np.array([0, 1, 2, 2, 5], dtype=np.int32)
    offs = np.array([0, 3, 5], dtype=np.int64)
    lams = np.array([0.3, 0.2], dtype=np.float64)
    ent = (accord.AccordPathEntry * 4)()

    def path(r, of, ns, lm, nl, n=10, p=10):
        return lib.accord_path(dummy, n, p, r.ctypes.data, of.ctypes.data, ns, lm.ctypes.data, nl, ctypes.byref(o),
                               ent, None, None, None, None, 0, ctypes.byref(st))
    assert path(rows, offs, 2, lams, 2, n=5) == accord.EINVAL          # row index 5 >= n
    assert path(rows, np.array([0, 3, 3], dtype=np.int64), 2, lams, 2) == accord.EINVAL  # empty subsample
    assert path(rows, offs, 2, np.array([0.3, -1.0]), 2) == accord.EINVAL  # negative penalty
    assert path(rows, offs, 0, lams, 2) == accord.EINVAL
    assert lib.accord_path_workspace_bytes(10, 10, rows.ctypes.data, offs.ctypes.data, 2, 2, ctypes.byref(o)) > 0
    assert lib.accord_path_workspace_bytes(5, 10, rows.ctypes.data, offs.ctypes.data, 2, 2, ctypes.byref(o)) == 0
    # post-processing and differentiation: argument checks before any device call
    assert lib.accord_postprocess(0, dummy, ctypes.byref(o), dummy, None) == accord.EINVAL
    assert lib.accord_postprocess(10, dummy, ctypes.byref(o), None, None) == accord.EINVAL
    assert lib.accord_grad_x(dummy, 10, 10, dummy, ctypes.byref(o), None) == accord.EINVAL
    d = ctypes.c_double()
    assert lib.accord_dloss_dloglam(dummy, 10, None, 5, 10, dummy, 0.2, ctypes.byref(o), ctypes.byref(d),
                                    None, None) == accord.EINVAL
    assert lib.accord_dloss_dloglam(dummy, 10, dummy, 5, 10, dummy, -0.2, ctypes.byref(o), ctypes.byref(d),
                                    None, None) == accord.EINVAL
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert accord.accord_status_string(s)


def test_binding_rejects_bad_arguments_on_the_host(lib):
    """The Python binding checks tensors before any device call: CPU tensors,
    wrong dtypes and shapes, unknown precision names."""
    import torch
    from paper_2412_11554_gb300 import accord
    X = torch.zeros(4, 6)
    with pytest.raises(ValueError):
        accord.accord_fit(X, 0.1)                           # not a CUDA tensor
    with pytest.raises(ValueError):
        accord.accord_fit(X.double(), 0.1)                  # float64 X needs precision="fp64" (and CUDA)
    with pytest.raises(KeyError):
        accord.accord_fit(X, 0.1, precision="fp16")         # no such mode
    with pytest.raises(ValueError):
        accord.accord_to_csr(torch.zeros(3, 4))             # not square, not CUDA
    with pytest.raises(ValueError):
        accord.accord_postprocess(torch.zeros(3, 3))        # not CUDA
    assert set(accord.PRECISIONS) == {"fp64", "mixed", "bf16x3", "tf32x3"}


def test_tensor_validator_on_host_tensors():
    """The binding's validator reports dtype, shape and layout mistakes before
    the device check, so each shows up here on host tensors."""
    import torch
    from paper_2412_11554_gb300 import accord
    chk = accord._check_tensor
    with pytest.raises(ValueError, match="torch.Tensor"):
        chk(np.zeros((3, 3)), "Omega", torch.float64)
    with pytest.raises(ValueError, match="must be torch.float64"):
        chk(torch.zeros(3, 3), "Omega", torch.float64, (3, 3))
    with pytest.raises(ValueError, match=r"shape \(3, 3\)"):
        chk(torch.zeros(3, 4, dtype=torch.float64), "Omega", torch.float64, (3, 3))
    with pytest.raises(ValueError, match="2-D"):
        chk(torch.zeros(12), "X", torch.float32, ndim=2)
    with pytest.raises(ValueError, match="contiguous"):
        chk(torch.zeros(4, 4).t()[:, :3], "X", torch.float32, ndim=2)
    with pytest.raises(ValueError, match="CUDA"):
        chk(torch.zeros(3, 3), "Omega", (torch.float32, torch.float64), (3, 3))
    assert accord._omega_dtype(accord.FP64) == torch.float64
    assert accord._omega_dtype(accord.MIXED_BF16X3) == accord._omega_dtype(accord.MIXED_TF32X3) == torch.float32
    assert accord._precision_of(None, torch.zeros(2, 2, dtype=torch.float64)) == accord.FP64
    assert accord._precision_of(None, torch.zeros(2, 2)) == accord.MIXED_BF16X3
    assert accord._precision_of("tf32x3", torch.zeros(2, 2, dtype=torch.float64)) == accord.MIXED_TF32X3


def test_binding_validates_every_caller_tensor(monkeypatch):
    """Every tensor a caller passes goes through the validator, with the dtype
    and shape the precision mode fixes, before the library sees its pointer.
    Recorded on the host with a fake library; the real validator then rejects
    any mismatch, a host tensor or another device."""
    import torch
    from paper_2412_11554_gb300 import accord
    seen = {}

    def record(t, name, dtype, shape=None, ndim=None):
        seen[t.data_ptr()] = (name, dtype if isinstance(dtype, tuple) else (dtype,), shape)

    calls = []

    class FakeLib:
        def __getattr__(self, fn):
            def call(*args):
                calls.append(fn)
                return 0
            return call

    class Stream:
        cuda_stream = 0

    monkeypatch.setattr(accord, "_check_tensor", record)
    monkeypatch.setattr(accord, "load_library", lambda path=None: FakeLib())
    n, p = 6, 4
    X, Xv, X64 = torch.zeros(n, p), torch.zeros(3, p), torch.zeros(n, p, dtype=torch.float64)
    O32, O64 = torch.zeros(p, p), torch.zeros(p, p, dtype=torch.float64)
    O32b, G32, GX = torch.zeros(p, p), torch.zeros(p, p), torch.zeros(n, p)
    fg, ws = torch.zeros(2, dtype=torch.float64), torch.zeros(64, dtype=torch.uint8)
    f32, f64, both = (torch.float32,), (torch.float64,), (torch.float32, torch.float64)
    S = Stream()
    cases = [
        ("accord_fit", lambda: accord.accord_fit(X, 0.1, Omega=O32, workspace=ws, stream=S),
         {X: f32, O32: f32, ws: (torch.uint8,)}),
        ("accord_fit", lambda: accord.accord_fit(X, 0.1, precision="fp64", Omega=O64, stream=S), {X: f32, O64: f64}),
        ("accord_refit", lambda: accord.accord_refit(X, 0.1, 0.5, O32, Omega=O32b, stream=S),
         {X: f32, O32: f32, O32b: f32}),
        ("accord_loss", lambda: accord.accord_loss(X, O32, 0.1, precision="fp64", stream=S), {X: f32, O32: f64}),
        ("accord_grad", lambda: accord.accord_grad(X, O32, out=G32, stream=S), {X: f32, O32: f32, G32: f32}),
        ("accord_grad", lambda: accord.accord_grad(X, O64, precision="tf32x3", stream=S), {X: f32, O64: f32}),
        ("accord_loss_f64_noalloc", lambda: accord.accord_loss_f64_noalloc(X64, O64, 0.1, fg, stream=S),
         {X64: f64, O64: f64, fg: f64}),
        ("accord_postprocess", lambda: accord.accord_postprocess(O32, stream=S), {O32: both}),
        ("accord_to_csr", lambda: accord.accord_to_csr(O64, stream=S), {O64: both}),
        ("accord_grad_x", lambda: accord.accord_grad_x(X, O32, out=GX, stream=S), {X: f32, O32: f32, GX: f32}),
        ("accord_dloss_dloglam", lambda: accord.accord_dloss_dloglam(X, Xv, O64, 0.1, precision="mixed", stream=S),
         {X: f32, Xv: f32, O64: f32}),
        ("accord_path", lambda: accord.accord_path(X, [np.arange(3)], [0.1], workspace=ws, stream=S),
         {X: f32, ws: (torch.uint8,)}),
    ]
    for fn, run, want in cases:
        seen.clear()
        calls.clear()
        run()
        assert fn in calls, fn
        for t, dts in want.items():
            assert t.data_ptr() in seen, (fn, t.shape)
            assert seen[t.data_ptr()][1] == dts, (fn, seen[t.data_ptr()])
        # square p x p operands are checked at that shape
        for t in (O32, O64, O32b, G32):
            if t.data_ptr() in seen and seen[t.data_ptr()][2] is not None:
                assert tuple(seen[t.data_ptr()][2]) == (p, p), fn


def test_largest_single_gpu_fit_sizes(lib):
    """The size limits the header states: at n = 1000 the workspace plus the
    caller's Omega and X fit a 284 GB GB300 (nvidia-smi's 284208 MiB, 3 % kept
    free) at p = 131000 (BF16x3), 117000 (TF32x3) and 108000 (FP64), and no
    longer at p 3 % larger."""
    from paper_2412_11554_gb300 import accord
    hbm = 0.97 * 284208 * 2 ** 20
    for prec, es, p_max, per_p2 in (("bf16x3", 4, 131000, 12.6), ("tf32x3", 4, 117000, 16.8),
                                    ("fp64", 8, 108000, 16.4)):
        def need(p):
            return accord.accord_workspace_bytes(1000, p, precision=prec) + es * p * p + 4 * 1000 * p
        assert need(p_max) <= hbm < need(int(p_max * 1.03)), prec
        # the per-p^2 growth quoted in the header
        per = accord.accord_workspace_bytes(1000, p_max, precision=prec) / p_max ** 2
        assert abs(per - per_p2) < 0.1, (prec, per)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every binding call raises; nothing falls
    back to another implementation."""
    import torch
    from paper_2412_11554_gb300 import accord
    monkeypatch.setattr(accord, "_LIB_PATH", str(tmp_path / "libaccord.so"))
    monkeypatch.setattr(accord, "_lib", None)
    for call in (lambda: accord.accord_default_opts(),
                 lambda: accord.accord_workspace_bytes(10, 10),
                 lambda: accord.accord_fit(torch.zeros(4, 6), 0.1),
                 lambda: accord.accord_status_string(0)):
        with pytest.raises(RuntimeError, match="libaccord.so not found"):
            call()


def test_path_sizing_needs_no_memory_in_n(lib):
    """Subsample bookkeeping grows with the subsamples, not with n: a data
    set of 2^40 rows sizes like one of 10 (run in a child process, which an
    abort would end alone), and repeated rows count once, so a bootstrap
    sample sizes like its distinct rows."""
    code = r'''
import ctypes, numpy as np
from paper_2412_11554_gb300 import accord
lib = accord.load_library()
o = accord.accord_default_opts()
def size(n, rows, offs):
    rows = np.asarray(rows, dtype=np.int32); offs = np.asarray(offs, dtype=np.int64)
    return lib.accord_path_workspace_bytes(n, 50, rows.ctypes.data, offs.ctypes.data, len(offs) - 1, 4, ctypes.byref(o))
big = size(1 << 40, [0, 1, 2, 7], [0, 4])
small = size(10, [0, 1, 2, 7], [0, 4])
boot = size(10, [2, 2, 0, 7, 1, 7, 7, 0], [0, 8])
distinct = size(10, [0, 1, 2, 7], [0, 4])
two = size(10, [3, 3, 3, 1, 0, 9], [0, 3, 6])
two_distinct = size(10, [3, 0, 1, 9], [0, 1, 4])
print(big, small, boot, distinct, two, two_distinct)
assert big == small > 0 and boot == distinct and two == two_distinct > 0
assert size(10, [0, 10], [0, 2]) == 0 and size(10, [0, -1], [0, 2]) == 0
'''
    import subprocess
    import sys
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr[-2000:])


def test_header_documents_each_computing_entry_point():
    """Each entry point that computes something cites the passage defining it
    and states its error behaviour in the comment above its declaration."""
    src = open(HEADER).read()
    docs = {m.group(3): m.group(1) for m in re.finditer(
        r"(/\*(?:(?!\*/).)*\*/)\s*((?:int|size_t)\s+(accord_\w+)\s*\([^;]*\);)", src, re.S)}
    computing = ["accord_fit", "accord_refit", "accord_fit_f64", "accord_loss", "accord_grad", "accord_grad_x",
                 "accord_dloss_dloglam", "accord_postprocess", "accord_to_csr", "accord_path",
                 "accord_path_workspace_bytes", "accord_workspace_bytes", "accord_loss_f64_noalloc"]
    cite = re.compile(r"Eq\. ?3\.\d|Sec \d|Algorithm \d|Thm \d|as accord_loss|as accord_fit")
    errs = re.compile(r"Errors|EINVAL|ENOMEM|EUNSUPPORTED|Returns|returns|0 on invalid|0 for invalid")
    for name in computing:
        assert name in docs, name
        assert cite.search(docs[name]), f"{name}: no passage cited"
        assert errs.search(docs[name]), f"{name}: no error behaviour"


def test_binding_constants_match_the_header():
    """Status codes, precision modes and trace columns of the binding equal
    the header's #defines."""
    from paper_2412_11554_gb300 import accord
    defs = dict(re.findall(r"#define\s+(ACCORD_\w+)\s+(-?\d+)", open(HEADER).read()))
    for name, val in (("OK", accord.OK), ("NOT_CONVERGED", accord.NOT_CONVERGED), ("EINVAL", accord.EINVAL),
                      ("EDOMAIN", accord.EDOMAIN), ("ENONFINITE", accord.ENONFINITE),
                      ("EBACKTRACK", accord.EBACKTRACK), ("ENOMEM", accord.ENOMEM), ("ECUDA", accord.ECUDA),
                      ("EUNSUPPORTED", accord.EUNSUPPORTED), ("FP64", accord.FP64),
                      ("MIXED_BF16X3", accord.MIXED_BF16X3), ("MIXED_TF32X3", accord.MIXED_TF32X3),
                      ("TRACE_FIELDS", accord.TRACE_FIELDS)):
        assert int(defs["ACCORD_" + name]) == val, name
    for col in ("f", "kkt", "tau", "ntrials", "nnz", "delta", "g"):
        assert int(defs["ACCORD_TRACE_" + col.upper()]) == accord.TRACE_COLUMNS.index(col), col


def test_testing_hooks_check_their_arguments_on_the_host(lib):
    """The two testing hooks only set process-wide values for later launches:
    out-of-range values are rejected and the defaults restored, all without a
    device."""
    from paper_2412_11554_gb300 import accord
    try:
        assert lib.accord_test_wait_limit(-1, 0) == accord.EINVAL
        assert lib.accord_test_wait_limit(0, 2) == accord.EINVAL
        for cap, form in ((31, 0), (513, 0), (0, -1), (0, 3), (-5, 1)):
            assert lib.accord_test_refresh(cap, form) == accord.EINVAL, (cap, form)
        for cap, form in ((32, 1), (512, 2), (0, 1)):
            assert lib.accord_test_refresh(cap, form) == accord.OK, (cap, form)
    finally:
        assert lib.accord_test_refresh(0, 0) == accord.OK
        assert lib.accord_test_wait_limit(0, 0) == accord.OK
