"""The C ABI on the host: the library builds, loads without a GPU, exports
every function include/sps.h declares, and rejects bad arguments before any
device work."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1901_00654_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sps.h")


@pytest.fixture(scope="module")
def B():
    build.build_library()
    from paper_1901_00654_gb300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SPS_API\s+[\w\s\*]+?\b(sps_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(B):
    names = declared_functions()
    assert len(names) >= 20
    lib = C.CDLL(build.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTED) == names


def test_struct_layouts_match_header(B):
    """sizeof/offsetof of the ABI structs from a C compiler equal the ctypes view."""
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "sps.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(sps_options), offsetof(sps_options, replace_ratio),
         offsetof(sps_options, precondition), offsetof(sps_options, lanes_r), sizeof(sps_result),
         offsetof(sps_result, solve_ms), offsetof(sps_options, coarse_iters), offsetof(sps_options, max_device_bytes),
         sizeof(sps_batch_shape));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [C.sizeof(B.sps_options), B.sps_options.replace_ratio.offset, B.sps_options.precondition.offset,
                    B.sps_options.lanes_r.offset, C.sizeof(B.sps_result), B.sps_result.solve_ms.offset,
                    B.sps_options.coarse_iters.offset, B.sps_options.max_device_bytes.offset,
                    C.sizeof(B.sps_batch_shape)]


def test_defaults(B):
    o = B.sps_default_options()
    assert (o.precision, o.nu1, o.nu2, o.omega, o.max_iter) == (B.SPS_PREC_FP64, 1, 1, 0.0, 20000)
    assert (o.hybrid, o.graphs, o.precondition, o.autotune, o.lanes_r) == (1, 1, 1, 0, 0)
    assert (o.coarse_cg, o.coarse_iters, o.max_device_bytes) == (0, 32, 0)


@pytest.mark.parametrize("args", [
    dict(P=0, intervals=[8]),
    dict(P=6, intervals=[8] * 6),
    dict(P=2, intervals=[8, 12]),
    dict(P=2, intervals=[8, 8], q=2),
    dict(P=2, intervals=[8, 8], levels=5),
    dict(P=2, intervals=[8, 8], lam=-1.0),
    dict(P=2, intervals=[8, 8], lam=float("nan")),
    dict(P=3, intervals=[1024, 1024, 1024]),
    dict(P=2, intervals=[8, 8], lo=[0.0, 1.0], hi=[1.0, 1.0]),
    dict(P=5, intervals=[16] * 5, levels=1),
])
def test_plan_create_rejects_bad_arguments(B, args):
    a = dict(q=3, levels=2, lam=1e-3, lo=None, hi=None)
    a.update(args)
    P = a["P"]
    h = C.c_void_p()
    iv = (C.c_int * max(P, 1))(*a["intervals"][:max(P, 1)])
    lo = (C.c_double * P)(*a["lo"]) if a["lo"] else None
    hi = (C.c_double * P)(*a["hi"]) if a["hi"] else None
    code = B.lib().sps_plan_create(C.byref(h), P, a["q"], iv, lo, hi, a["levels"], a["lam"], None)
    assert code == B.SPS_EINVAL
    assert h.value is None
    assert len(B.sps_last_error()) > 0


def test_null_handles(B):
    assert B.lib().sps_destroy(None) == B.SPS_OK
    assert B.lib().sps_solve(None, None, 0, 1e-8, None, None) == B.SPS_EINVAL
    assert B.lib().sps_set_points(None, 10, None, None, 1, 0, None) == B.SPS_EINVAL
    assert B.lib().sps_get_tuning(None, 1, None, None) == B.SPS_EINVAL
    assert B.lib().sps_launch_count(None) == B.SPS_EINVAL


@pytest.mark.parametrize("field,value", [("autotune", 2), ("lanes_r", 1), ("lanes_r", 4), ("tile", 3),
                                         ("coarse_cg", 3), ("coarse_iters", 0)])
def test_plan_create_rejects_bad_options(B, field, value):
    o = B.sps_default_options()
    setattr(o, field, value)
    h = C.c_void_p()
    iv = (C.c_int * 2)(8, 8)
    assert B.lib().sps_plan_create(C.byref(h), 2, 3, iv, None, None, 2, 1e-3, C.byref(o)) == B.SPS_EINVAL
    assert h.value is None


def test_evaluate_rejects_bad_arguments(B):
    assert B.lib().sps_evaluate(None, None, 0, None, 1, None, 0, None) == B.SPS_EINVAL
    o = B.sps_default_options()
    h = C.c_void_p()
    iv = (C.c_int * 2)(8, 8)
    # plan creation and argument checks run before any device work
    if B.lib().sps_plan_create(C.byref(h), 2, 3, iv, None, None, 2, 1e-3, C.byref(o)) != B.SPS_OK:
        pytest.skip("plan creation needs a GPU here")
    try:
        assert B.lib().sps_evaluate(h, None, -1, None, 1, None, 0, None) == B.SPS_EINVAL
        assert B.lib().sps_evaluate(h, None, 4, None, 1, None, 0, None) == B.SPS_EINVAL
        assert B.lib().sps_evaluate(h, None, 0, None, 7, None, 0, None) == B.SPS_EINVAL
    finally:
        B.lib().sps_destroy(h)


def _lanczos(S, m, seed):
    """m steps of the plain Lanczos recurrence on the symmetric matrix S
    (no reorthogonalisation, as the library runs it): alpha_j and beta_j^2."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(S.shape[0])
    q /= np.linalg.norm(q)
    qp = np.zeros_like(q)
    a, b2, beta = [], [], 0.0
    for _ in range(m):
        w = S @ q
        alpha = q @ w
        w = w - alpha * q - beta * qp
        a.append(alpha)
        b2.append(w @ w)
        beta = np.sqrt(b2[-1])
        qp, q = q, (w / beta if beta > 0 else np.zeros_like(w))
    return np.array(a), np.array(b2)


@pytest.mark.parametrize("n, m", [(12, 12), (300, 20), (300, 32), (5, 1)])
def test_lanczos_estimate_of_the_damping(B, n, m):
    """Host logic of omega_g (no GPU): the top Ritz value equals the largest
    eigenvalue of the Lanczos tridiagonal T_m (numpy), the estimate adds the
    Ritz residual beta_m |s_m| so that it bounds lambda_max(S) once the Ritz
    value has converged, and with m = n (an invariant Krylov space) it is
    lambda_max itself."""
    rng = np.random.default_rng(n + m)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.concatenate([[2.0], rng.uniform(0.05, 1.7, n - 1)])   # a gap below lambda_max = 2
    S = (Q * ev) @ Q.T
    a, b2 = _lanczos(S, m, seed=n)
    theta, lhat = B.sps_lanczos_estimate(a, b2)
    b = np.sqrt(b2)
    T = np.diag(a) + np.diag(b[:m - 1], 1) + np.diag(b[:m - 1], -1)
    w, V = np.linalg.eigh(T)
    assert abs(theta - w[-1]) <= 1e-12 * abs(w[-1])
    assert abs(lhat - (w[-1] + b[m - 1] * abs(V[-1, -1]))) <= 1e-9 * w[-1]
    if m == n:
        assert abs(theta - 2.0) < 1e-9 and abs(lhat - 2.0) < 1e-6
    if m >= 20:
        assert 2.0 <= lhat * (1 + 1e-12) and lhat < 2.0 * 1.05


def test_lanczos_estimate_rejects_bad_input(B):
    with pytest.raises(B.SpsError):
        B.sps_lanczos_estimate(np.zeros(0), np.zeros(0))
    with pytest.raises(B.SpsError):
        B.sps_lanczos_estimate(np.ones(33), np.ones(33))
    with pytest.raises(B.SpsError):
        B.sps_lanczos_estimate(np.array([np.nan]), np.array([1.0]))
    with pytest.raises(B.SpsError):
        B.sps_lanczos_estimate(np.array([-1.0]), np.array([0.0]))
