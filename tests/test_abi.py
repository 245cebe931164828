"""C ABI checks that need no GPU: the library builds and loads, exports every
function the header declares, and the ctypes mirrors of the structs have the
same sizes and field offsets as the C compiler gives them."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2204_08183_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "survgpu.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return [n for n in names if n not in ("if", "while", "return")]


def test_header_functions_are_exported(libpath):
    declared = _declared_functions()
    assert "cox_fit" in declared and "fg_fit" in declared and "loglik_grad_hess" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert sorted(declared) == sorted(binding.EXPORTS)


def test_library_loads_without_gpu(libpath):
    lib = C.CDLL(libpath)
    for name in binding.EXPORTS:
        assert hasattr(lib, name)
    lib.surv_version.restype = C.c_int
    assert lib.surv_version() >= 100
    lib.surv_strerror.restype = C.c_char_p
    assert lib.surv_strerror(-2) == b"time not sorted in decreasing order"


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "survgpu.h"
#define F(S, m) printf(#S "." #m " %zu\n", offsetof(S, m))
int main(void) {
  printf("surv_data %zu\n", sizeof(surv_data));
  printf("surv_opts %zu\n", sizeof(surv_opts));
  printf("surv_fit_info %zu\n", sizeof(surv_fit_info));
  printf("surv_nll_data %zu\n", sizeof(surv_nll_data));
  printf("surv_cv_info %zu\n", sizeof(surv_cv_info));
  F(surv_cv_info, nfits); F(surv_cv_info, best_lambda); F(surv_cv_info, max_sweeps_used);
  F(surv_cv_info, fits_converged); F(surv_cv_info, graph_replays); F(surv_cv_info, ctas_per_fit);
  F(surv_cv_info, row_pass_form); F(surv_cv_info, tile_form);
  F(surv_cv_info, kernel_launches); F(surv_cv_info, n_groups); F(surv_cv_info, coordinate_passes);
  F(surv_cv_info, eta_updates); F(surv_cv_info, ccd_kernel_ms);
  F(surv_cv_info, heldout_ms);
  F(surv_nll_data, n); F(surv_nll_data, p); F(surv_nll_data, ncols); F(surv_nll_data, time);
  F(surv_nll_data, status); F(surv_nll_data, X);
  F(surv_data, n); F(surv_data, p); F(surv_data, time); F(surv_data, status); F(surv_data, layout);
  F(surv_data, dtype); F(surv_data, col_ptr); F(surv_data, row_idx); F(surv_data, values);
  F(surv_opts, penalty); F(surv_opts, precision); F(surv_opts, lambda); F(surv_opts, penalty_factor);
  F(surv_opts, tol); F(surv_opts, max_sweeps); F(surv_opts, flags); F(surv_opts, wait_limit_s);
  F(surv_opts, stream); F(surv_opts, workspace);
  F(surv_fit_info, sweeps); F(surv_fit_info, converged); F(surv_fit_info, nnz_beta);
  F(surv_fit_info, device_error); F(surv_fit_info, loglik); F(surv_fit_info, objective);
  F(surv_fit_info, objective_prev); F(surv_fit_info, n_groups); F(surv_fit_info, coordinate_passes);
  F(surv_fit_info, eta_updates); F(surv_fit_info, kernel_launches); F(surv_fit_info, ccd_kernel_ms); F(surv_fit_info, phase_ms);
  F(surv_fit_info, row_passes);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c = dict(line.split() for line in out if line.strip())
    structs = {"surv_data": binding.surv_data, "surv_opts": binding.surv_opts,
               "surv_fit_info": binding.surv_fit_info, "surv_nll_data": binding.surv_nll_data,
               "surv_cv_info": binding.surv_cv_info}
    for name, cls in structs.items():
        assert int(c[name]) == C.sizeof(cls), name
    for key, off in c.items():
        if "." not in key:
            continue
        sname, field = key.split(".")
        field = "lambda_" if field == "lambda" else field
        assert getattr(structs[sname], field).offset == int(off), key


def test_library_reads_no_environment_knobs():
    # every schedule choice goes through surv_opts.flags
    csrc = os.path.join(ROOT, "paper_2204_08183_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "getenv" not in open(os.path.join(csrc, f)).read(), f


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2204_08183_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    # no CPU fallback: a missing library is an error, not a silent substitute
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="libsurvgpu.so not found"):
        binding.load(str(tmp_path / "libsurvgpu.so"))


def test_header_documents_every_flag_the_binding_uses():
    text = open(HEADER).read()
    for name in ("SURV_FLAG_TEST_STALL", "SURV_FLAG_PERSISTENT", "SURV_FLAG_CV_TUNE", "SURV_FLAG_SPARSE_NUMERATOR",
                 "SURV_FLAG_ONE_COORDINATE", "SURV_FLAG_SPEC_B8", "SURV_FLAG_NO_PDL",
                 "SURV_FLAG_CV_TILE1", "SURV_FLAG_CV_TILE2"):
        m = re.search(r"#define %s (\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(binding, name), name


def test_survdata_host_checks():
    """Marshalling checks that run before any library call."""
    import numpy as np
    import torch
    from paper_2204_08183_gb300 import binding
    n, p = 64, 3
    t = np.arange(n, 0, -1, dtype=np.int32)
    s = np.ones(n, np.int8)
    Xf = np.asfortranarray(np.ones((n, p), np.float32))
    d = binding.SurvData(t, s, X=Xf)
    assert (d.n, d.p, d.c.layout, d.c.dtype) == (n, p, binding.SURV_DENSE, binding.SURV_F32)
    with pytest.raises(ValueError):
        binding.SurvData(t, s, X=np.ascontiguousarray(Xf))          # C order is not column-major
    with pytest.raises(ValueError):
        binding.SurvData(t, s, X=torch.ones(n, p))                   # torch X must be (p, n)
    d = binding.SurvData(t, s, X=torch.ones(p, n, dtype=torch.bfloat16))
    assert d.c.dtype == binding.SURV_BF16 and d.p == p
    with pytest.raises(TypeError):
        binding.SurvData(t, s, X=np.asfortranarray(np.ones((n, p), np.int32)))
    with pytest.raises(ValueError):
        binding.SurvData(t, s, X=torch.ones(2 * p, n)[::2])          # not contiguous
    cp = np.array([0, 2, 2, 4], np.int64)
    ri = np.array([0, 5, 1, 7], np.int32)
    d = binding.SurvData(t, s, col_ptr=cp, row_idx=ri)
    assert (d.p, d.c.layout, d.c.dtype, d.c.values) == (3, binding.SURV_CSC, binding.SURV_F32, None)
    d = binding.SurvData(t, s, col_ptr=cp, row_idx=ri, values=np.ones(4, np.float64))
    assert d.c.dtype == binding.SURV_F64


def test_argument_errors_before_any_device_call(libpath):
    """Argument checks of the fits, the evaluation, lambda_max and the CV
    path return their codes before the first CUDA call, so they hold on a
    host without a GPU too."""
    import numpy as np
    n = 50
    t = np.arange(n, 0, -1, dtype=np.int32)
    s = np.ones(n, np.int8)
    cp = np.array([0, 3, 5], np.int64)
    ri = np.array([1, 4, 9, 2, 3], np.int32)
    good = binding.SurvData(t, s, col_ptr=cp, row_idx=ri)
    beta = np.zeros(2)

    def code(fn, *a, **kw):
        with pytest.raises(binding.SurvError) as ei:
            fn(*a, **kw)
        return ei.value.code

    E = binding
    # sizes, layout, dtype
    nop = binding.SurvData(t, s, col_ptr=np.zeros(1, np.int64), row_idx=ri)
    assert code(binding.cox_fit, nop, beta=np.zeros(1)) == E.SURV_E_INVALID
    bfc = binding.SurvData(t, s, col_ptr=cp, row_idx=ri, values=np.zeros(5, np.float32))
    bfc.c.dtype = binding.SURV_BF16                       # bfloat16 is for dense X only
    assert code(binding.cox_fit, bfc, beta=beta) == E.SURV_E_INVALID
    bad_layout = binding.SurvData(t, s, col_ptr=cp, row_idx=ri)
    bad_layout.c.layout = 7
    assert code(binding.fg_fit, bad_layout, beta=beta) == E.SURV_E_INVALID
    empty = binding.SurvData(t[:0], s[:0], col_ptr=np.zeros(3, np.int64), row_idx=ri[:0])
    assert code(binding.cox_fit, empty, beta=beta) == E.SURV_E_NO_EVENTS
    # options
    assert code(binding.cox_fit, good, beta=beta, penalty="l1", lam=-1.0) == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, lam=float("nan")) == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, tol=-1.0) == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, max_sweeps=-1) == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, flags=1 << 20) == E.SURV_E_INVALID
    # the sparse-numerator form is for Cox fits of CSC data in the FP32 mode
    sn = binding.SURV_FLAG_SPARSE_NUMERATOR
    assert code(binding.fg_fit, good, beta=beta, flags=sn) == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, flags=sn, precision="f64") == E.SURV_E_INVALID
    assert code(binding.cox_fit, good, beta=beta, flags=sn | binding.SURV_FLAG_PERSISTENT) == E.SURV_E_INVALID
    # single evaluation: coordinate out of range
    assert code(binding.loglik_grad_hess, good, "cox", beta, 2) == E.SURV_E_INVALID
    # CV path: fold and lambda counts, flags
    fold = np.zeros(n, np.int8)
    lam = np.ones(3)
    assert code(binding.cox_cv_path, good, fold, 0, lam) == E.SURV_E_INVALID
    assert code(binding.cox_cv_path, good, fold, 128, lam) == E.SURV_E_INVALID
    assert code(binding.cox_cv_path, good, fold, 2, lam, ctas_per_fit=-1) == E.SURV_E_INVALID
    both = binding.SURV_FLAG_CV_TILE1 | binding.SURV_FLAG_CV_TILE2        # two tile shapes at once
    assert code(binding.cox_cv_path, good, fold, 2, lam, flags=both) == E.SURV_E_INVALID
    assert code(binding.cox_cv_path, good, fold, 2, lam, flags=binding.SURV_FLAG_ONE_COORDINATE) == E.SURV_E_INVALID
    assert code(binding.cox_cv_path, empty, fold, 2, lam) == E.SURV_E_NO_EVENTS
    # lambda_max checks the data first
    assert code(binding.cox_lambda_max, bad_layout) == E.SURV_E_INVALID


def test_noalloc_argument_errors_before_any_device_call(libpath):
    """loglik_grad_hess_noalloc rejects out-of-range sizes, a bad coordinate,
    values whose dtype differs from the precision and misaligned dense X
    before its first CUDA call."""
    import numpy as np
    n = 40
    t = np.arange(n, 0, -1, dtype=np.int32)
    s = np.ones(n, np.int8)

    def code(*a, **kw):
        with pytest.raises(binding.SurvError) as ei:
            binding.loglik_grad_hess_noalloc(*a, **kw)
        return ei.value.code

    E = binding
    wide = 4097                                              # more covariates than the limit
    cpw = np.zeros(wide + 1, np.int64)
    dw = binding.SurvData(t, s, col_ptr=cpw, row_idx=np.zeros(1, np.int32), p=wide)
    assert code(dw, "cox", np.zeros(wide), 0) == E.SURV_E_INVALID
    cp = np.array([0, 3, 5], np.int64)
    ri = np.array([1, 4, 9, 2, 3], np.int32)
    good = binding.SurvData(t, s, col_ptr=cp, row_idx=ri)
    assert code(good, "cox", np.zeros(2), 2) == E.SURV_E_INVALID           # j out of range
    assert code(good, "cox", np.zeros(2), -1) == E.SURV_E_INVALID
    f64 = binding.SurvData(t, s, col_ptr=cp, row_idx=ri, values=np.ones(5, np.float64))
    assert code(f64, "cox", np.zeros(2), 0) == E.SURV_E_INVALID             # float64 values, FP32 mode
    X = np.asfortranarray(np.ones((n, 2), np.float32))
    assert code(binding.SurvData(t, s, X=X), "cox", np.zeros(2), 0, precision="f64") == E.SURV_E_INVALID
    n3 = 39                                                  # dense X needs n divisible by 4
    d3 = binding.SurvData(t[:n3], s[:n3], X=np.asfortranarray(np.ones((n3, 2), np.float32)))
    assert code(d3, "cox", np.zeros(2), 0) == E.SURV_E_INVALID
    buf = np.zeros(2 * n + 4, np.float32)
    mis = buf[1:1 + 2 * n].reshape(2, n).T                   # 4-byte offset base: not 16-byte aligned
    assert mis.flags["F_CONTIGUOUS"] and mis.ctypes.data % 16 != 0
    assert code(binding.SurvData(t, s, X=mis), "cox", np.zeros(2), 0) == E.SURV_E_INVALID


def test_nll_argument_errors_before_any_device_call(libpath):
    """cox_nll_forward / cox_nll_backward reject a column count outside
    1..64, host arrays, and a backward with no forward before it on the
    workspace, before their first CUDA call."""
    import torch
    n, p, C = 64, 8, 4
    X = torch.zeros((n, p), dtype=torch.bfloat16)
    t = torch.arange(n, 0, -1, dtype=torch.int32)
    s = torch.ones(n, dtype=torch.int8)
    ws = binding.Workspace()

    def code(fn, *a):
        with pytest.raises(binding.SurvError) as ei:
            fn(*a)
        return ei.value.code

    E = binding
    assert code(binding.cox_nll_forward, X, t, s, torch.zeros((p, 65), dtype=torch.float32), ws) == E.SURV_E_INVALID
    assert code(binding.cox_nll_forward, X, t, s, torch.zeros((p, 0), dtype=torch.float32), ws) == E.SURV_E_INVALID
    # host tensors: the arrays must be device memory
    assert code(binding.cox_nll_forward, X, t, s, torch.zeros((p, C), dtype=torch.float32), ws) == E.SURV_E_INVALID
    # no forward on this workspace yet
    g = torch.ones(C, dtype=torch.float64)
    assert code(binding.cox_nll_backward, X, t, s, g, C, ws) == E.SURV_E_INVALID


def test_sort_and_groups_argument_errors(libpath):
    """surv_sort_desc and surv_groups reject a negative n and null arrays (and
    surv_groups a null K) before any CUDA call; n = 0 is a no-op."""
    import ctypes
    import numpy as np
    lib = binding.load()
    t = np.arange(8, 0, -1, dtype=np.int32)
    s = np.ones(8, np.int8)
    perm = np.empty(8, np.int32)
    tp, sp, pp = (ctypes.c_void_p(a.ctypes.data) for a in (t, s, perm))
    K = ctypes.c_int64()
    E = binding
    assert lib.surv_sort_desc(tp, -1, pp, None) == E.SURV_E_INVALID
    assert lib.surv_sort_desc(None, 8, pp, None) == E.SURV_E_INVALID
    assert lib.surv_sort_desc(tp, 8, None, None) == E.SURV_E_INVALID
    assert lib.surv_sort_desc(tp, 0, pp, None) == E.SURV_OK
    assert lib.surv_groups(tp, sp, -1, 0, ctypes.byref(K), None, None, None, None) == E.SURV_E_INVALID
    assert lib.surv_groups(tp, sp, 8, 0, None, None, None, None, None) == E.SURV_E_INVALID
    assert lib.surv_groups(None, sp, 8, 0, ctypes.byref(K), None, None, None, None) == E.SURV_E_INVALID
    assert lib.surv_groups(tp, None, 8, 0, ctypes.byref(K), None, None, None, None) == E.SURV_E_INVALID
