"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function include/dcd_gb300.h declares, and the ctypes structures match the
header's layout (checked by compiling the header with gcc)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dcd_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["dcd_svm_solve", "bdcd_krr_solve", "dcd_status_string", "dcd_sample_indices", "dcd_kernel_block",
              "dcd_kernel_block_apply"]:
        assert f in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2406_18001_gb300 import binding
    L = binding.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(binding.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(r"\bT " + name + r"\b", out), name


def test_status_strings():
    from paper_2406_18001_gb300 import binding
    assert binding.status_string(0) == "DCD_OK"
    assert "invalid" in binding.status_string(1)
    assert "unknown" in binding.status_string(99)


LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "dcd_gb300.h"
#define F(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("dcd_matrix %zu\n", sizeof(dcd_matrix));
  printf("dcd_kernel %zu\n", sizeof(dcd_kernel));
  printf("dcd_opts %zu\n", sizeof(dcd_opts));
  printf("dcd_stats %zu\n", sizeof(dcd_stats));
  F(dcd_matrix, values); F(dcd_matrix, row_scale); F(dcd_kernel, gamma); F(dcd_kernel, coef0);
  F(dcd_opts, seed); F(dcd_opts, tol); F(dcd_opts, flags); F(dcd_stats, final_metric); F(dcd_stats, ms_check);
  F(dcd_stats, refreshes); F(dcd_stats, s_used);
  printf("dcd_krr_problem %zu\n", sizeof(dcd_krr_problem));
  printf("dcd_batch_opts %zu\n", sizeof(dcd_batch_opts));
  F(dcd_krr_problem, y); F(dcd_krr_problem, k); F(dcd_krr_problem, lambda); F(dcd_krr_problem, b);
  F(dcd_krr_problem, max_iters); F(dcd_krr_problem, alpha); F(dcd_krr_problem, grad);
  F(dcd_batch_opts, tol); F(dcd_batch_opts, flags);
  return 0;
}
"""


def test_ctypes_layout_matches_header(tmp_path):
    from paper_2406_18001_gb300 import binding as b
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.splitlines())
    assert int(got["dcd_matrix"]) == C.sizeof(b.Matrix)
    assert int(got["dcd_kernel"]) == C.sizeof(b.Kernel)
    assert int(got["dcd_opts"]) == C.sizeof(b.Opts)
    assert int(got["dcd_stats"]) == C.sizeof(b.Stats)
    assert int(got["dcd_matrix.values"]) == b.Matrix.values.offset
    assert int(got["dcd_matrix.row_scale"]) == b.Matrix.row_scale.offset
    assert int(got["dcd_kernel.gamma"]) == b.Kernel.gamma.offset
    assert int(got["dcd_kernel.coef0"]) == b.Kernel.coef0.offset
    assert int(got["dcd_opts.seed"]) == b.Opts.seed.offset
    assert int(got["dcd_opts.tol"]) == b.Opts.tol.offset
    assert int(got["dcd_opts.flags"]) == b.Opts.flags.offset
    assert int(got["dcd_stats.final_metric"]) == b.Stats.final_metric.offset
    assert int(got["dcd_stats.ms_check"]) == b.Stats.ms_check.offset
    assert int(got["dcd_stats.refreshes"]) == b.Stats.refreshes.offset
    assert int(got["dcd_stats.s_used"]) == b.Stats.s_used.offset
    assert int(got["dcd_krr_problem"]) == C.sizeof(b.KrrProblem)
    assert int(got["dcd_batch_opts"]) == C.sizeof(b.BatchOpts)
    for f, cf in (("y", "y"), ("k", "k"), ("lambda", "lam"), ("b", "b"), ("max_iters", "max_iters"),
                  ("alpha", "alpha"), ("grad", "grad")):
        assert int(got[f"dcd_krr_problem.{f}"]) == getattr(b.KrrProblem, cf).offset
    assert int(got["dcd_batch_opts.tol"]) == b.BatchOpts.tol.offset
    assert int(got["dcd_batch_opts.flags"]) == b.BatchOpts.flags.offset


def test_host_validation_rejects_bad_arguments_without_gpu():
    """Argument checks run on the host before any CUDA call."""
    from paper_2406_18001_gb300 import binding as b
    L = b.lib()
    A = np.zeros((4, 3))
    Am = b.dense_matrix(A)
    k = b.kernel("rbf", gamma=1.0)
    o = b._opts(1, 1, 10, 0, 0, 0.0, 0, "fp64", 0)
    y = np.ones(4)
    al = np.zeros(4)
    # C <= 0
    assert L.dcd_svm_solve(C.byref(Am), b._ptr(y), C.byref(k), 1, 0.0, C.byref(o), b._ptr(al), None, None,
                           None) == b.EINVAL
    # bad loss
    assert L.dcd_svm_solve(C.byref(Am), b._ptr(y), C.byref(k), 3, 1.0, C.byref(o), b._ptr(al), None, None,
                           None) == b.EINVAL
    # b != 1 for DCD
    o2 = b._opts(1, 2, 10, 0, 0, 0.0, 0, "fp64", 0)
    assert L.dcd_svm_solve(C.byref(Am), b._ptr(y), C.byref(k), 1, 1.0, C.byref(o2), b._ptr(al), None, None,
                           None) == b.EINVAL
    # lambda <= 0, b > m
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(k), -1.0, C.byref(o), b._ptr(al), None, None,
                            None) == b.EINVAL
    o3 = b._opts(1, 5, 10, 0, 0, 0.0, 0, "fp64", 0)
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(k), 1.0, C.byref(o3), b._ptr(al), None, None,
                            None) == b.EINVAL
    # bad kernels
    kb = b.kernel("rbf", gamma=-1.0)
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(kb), 1.0, C.byref(o), b._ptr(al), None, None,
                            None) == b.EINVAL
    kp = b.kernel("poly", coef0=-1.0, degree=3)
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(kp), 1.0, C.byref(o), b._ptr(al), None, None,
                            None) == b.EINVAL
    kp1 = b.kernel("poly", coef0=1.0, degree=1)
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(kp1), 1.0, C.byref(o), b._ptr(al), None, None,
                            None) == b.EINVAL
    # s*b too large, null arrays, reserved precisions
    o4 = b._opts(100000, 1, 10, 0, 0, 0.0, 0, "fp64", 0)
    assert L.dcd_svm_solve(C.byref(Am), b._ptr(y), C.byref(k), 1, 1.0, C.byref(o4), b._ptr(al), None, None,
                           None) == b.EINVAL
    assert L.dcd_svm_solve(None, b._ptr(y), C.byref(k), 1, 1.0, C.byref(o), b._ptr(al), None, None,
                           None) == b.EINVAL
    o5 = b._opts(1, 1, 10, 0, 0, 0.0, 0, "fp8", 0)
    assert L.dcd_svm_solve(C.byref(Am), b._ptr(y), C.byref(k), 1, 1.0, C.byref(o5), b._ptr(al), None, None,
                           None) == b.EUNSUPPORTED
    # the accurate split-tf32 epilogue is an apply-only precision
    o6 = b._opts(1, 1, 10, 0, 0, 0.0, 0, "refresh", 0)
    assert L.bdcd_krr_solve(C.byref(Am), b._ptr(y), C.byref(k), 1.0, C.byref(o6), b._ptr(al), None, None,
                            None) == b.EUNSUPPORTED
    cols = np.zeros(2, dtype=np.int32)
    out = np.zeros(8)
    for fn in (L.dcd_kernel_block, L.dcd_kernel_block_static):
        assert fn(C.byref(Am), C.byref(k), b.PREC_REFRESH, None, 4, b._ptr(cols), 2, b._ptr(out), 2,
                  None) == b.EUNSUPPORTED
    # sampler argument checks
    assert L.dcd_sample_indices(2, 0, 10, 1, 0, 5, None, None) == b.EINVAL
    assert L.dcd_sample_indices(1, 0, 10, 11, 0, 5, None, None) == b.EINVAL
