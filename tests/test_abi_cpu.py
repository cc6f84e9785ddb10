"""Host-side checks of libsto that need no GPU: it loads, exports every
symbol include/sto.h declares, and validates arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_2312_01121_b300 import build, sto

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sto.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sto.h")).read()
    return sorted(set(re.findall(r"^STO_API\s+[\w\s\*]*?\b(sto_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["sto_create", "sto_run", "sto_set_state", "sto_get_state", "sto_destroy",
                     "sto_strerror", "sto_default_params", "sto_create_ex"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sto.SIGNATURES), "binding and header disagree"


def test_exports_are_only_the_abi():
    out = os.popen(f"nm -D --defined-only {sto.LIB_PATH}").read()
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {n for n in exported if n.startswith("sto_")} == set(declared_symbols())


def test_abi_version_and_strerror(lib):
    assert lib.sto_abi_version() == 4
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert sto.sto_strerror(code)
    assert "invalid" in sto.sto_strerror(-1)
    assert "positive definite" in sto.sto_strerror(sto.STO_ESINGULAR)


def test_default_params_are_the_paper_table(lib):
    p = sto.sto_default_params()
    assert p == sto.Params()
    assert (p.gamma, p.alpha, p.Ms, p.Hk, p.Happl) == (1.764e7, 0.005, 1448.3, 18616.0, 200.0)
    assert (p.eta, p.lambda_, p.current, p.A_cp, p.A_in, p.dt) == (0.537, 0.288, 2.5e-3, 1.0, 1.0, 1e-11)
    assert p.p == (1.0, 0.0, 6.123234e-17)


def test_struct_layouts_match_the_header(tmp_path):
    """ctypes mirrors vs the C compiler's sizeof / offsetof of include/sto.h."""
    fields = {"sto_params": [f[0] for f in sto.sto_params._fields_],
              "sto_config": [f[0] for f in sto.sto_config._fields_],
              "sto_info": [f[0] for f in sto.sto_info._fields_],
              "sto_batch_plan": [f[0] for f in sto.sto_batch_plan._fields_],
              "sto_grads": [f[0] for f in sto.sto_grads._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sto.h"', "int main(void){"]
    for st, names in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for n in names:
            cn = "lambda" if n == "lambda_" else n
            lines.append(f'printf("{st}.{n} %zu\\n", offsetof({st}, {cn}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    assert os.system(f"gcc -I {ROOT}/include -o {exe} {src}") == 0
    got = dict(l.split() for l in os.popen(str(exe)).read().splitlines())
    for st, names in fields.items():
        cls = getattr(sto, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for n in names:
            assert int(got[f"{st}.{n}"]) == getattr(cls, n).offset, f"{st}.{n}"


def test_invalid_arguments_rejected_before_cuda(lib):
    cp = sto.Params().to_c()
    h = ctypes.c_void_p()
    buf = (ctypes.c_float * 4)()
    assert lib.sto_create(0, ctypes.byref(cp), buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_create(2, ctypes.byref(cp), None, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_create(2, None, buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_create(2, ctypes.byref(cp), buf, buf, None, None, None) == sto.STO_EINVAL
    bad = sto.Params(substeps=0).to_c()
    assert lib.sto_create(2, ctypes.byref(bad), buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    bad = sto.Params(dt=float("nan")).to_c()
    assert lib.sto_create(2, ctypes.byref(bad), buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    bad = sto.Params(sample_component=3).to_c()
    assert lib.sto_create(2, ctypes.byref(bad), buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    dbuf = (ctypes.c_double * 4)()
    for product in (0, 3, -1):
        assert lib.sto_create_f64(2, ctypes.byref(cp), dbuf, buf, None, None, None, product,
                                  ctypes.byref(h)) == sto.STO_EINVAL
    for product in (sto.STO_PRODUCT_DF, sto.STO_PRODUCT_F64):
        assert lib.sto_create_f64(0, ctypes.byref(cp), dbuf, buf, None, None, None, product,
                                  ctypes.byref(h)) == sto.STO_EINVAL
        assert lib.sto_create_f64(2, ctypes.byref(cp), None, buf, None, None, None, product,
                                  ctypes.byref(h)) == sto.STO_EINVAL
        assert lib.sto_create_f64(2, ctypes.byref(cp), dbuf, buf, None, None, None, product,
                                  None) == sto.STO_EINVAL
    assert lib.sto_run(None, buf, 1, None) == sto.STO_EINVAL
    assert lib.sto_get_info(None, None) == sto.STO_EINVAL
    lib.sto_destroy(None)
    b = ctypes.c_void_p()
    assert lib.sto_batch_create(2, 0, ctypes.byref(cp), None, None, buf, buf, None, None,
                                ctypes.byref(b)) == sto.STO_EINVAL
    # the sweep's update indexes its [3][R][N] state with 32-bit offsets: R N <= 2^29
    for N, R in ((32769, 1), (1, 65537), (20000, 30000)):
        assert lib.sto_batch_create(N, R, ctypes.byref(cp), None, None, buf, buf, None, None,
                                    ctypes.byref(b)) == sto.STO_ENOTSUP, (N, R)


def test_noalloc_wrapper_checks_extents_before_the_call(lib):
    """sto_run_noalloc reads and writes caller arrays in place and the C side
    cannot see their extents: the binding rejects short or mis-sized arrays
    with ValueError before the library is called (no GPU needed)."""
    import numpy as np
    N, T = 8, 3
    P = sto.Params(n_in=2)
    ok = {"W": np.zeros(N * N, np.float32), "w_in": np.zeros(N * 2, np.float32),
          "state": np.zeros(3 * N), "u": np.zeros(T * 2, np.float32),
          "states_out": np.zeros(T * N, np.float32)}
    bad = {"W": np.zeros(N * N - 1, np.float32), "w_in": np.zeros(N, np.float32),
           "state": np.zeros(3 * N + 1), "u": np.zeros(T * 2 - 1, np.float32),
           "states_out": np.zeros(T * N - 1, np.float32)}
    for name in ok:
        args = dict(ok)
        args[name] = bad[name]
        with pytest.raises(ValueError, match=name):
            sto.sto_run_noalloc(N, P, args["W"], args["w_in"], args["state"], args["u"], T,
                                args["states_out"])


def test_new_entry_points_reject_arguments_before_cuda(lib):
    """The readout, row-shard, group and single-launch sweep entry points
    check their arguments before any CUDA call (no GPU needed)."""
    buf = (ctypes.c_float * 64)()
    dbuf = (ctypes.c_double * 64)()
    out = ctypes.c_double()
    # readout: null pointers, empty or inverted ranges, negative ridge, N too large
    assert lib.sto_readout_fit(None, 4, 2, dbuf, 0, 4, 0.1, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_fit(buf, 4, 2, None, 0, 4, 0.1, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_fit(buf, 4, 2, dbuf, 0, 4, 0.1, None, None) == sto.STO_EINVAL
    for t0, t1 in ((-1, 2), (3, 3), (3, 2), (0, 5)):
        assert lib.sto_readout_fit(buf, 4, 2, dbuf, t0, t1, 0.1, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_fit(buf, 4, 2, dbuf, 0, 4, -1.0, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_fit(buf, 4, 2, dbuf, 0, 4, float("nan"), dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_fit(buf, 4, 40000, dbuf, 0, 4, 0.1, dbuf, None) == sto.STO_ENOTSUP
    assert lib.sto_readout_predict(buf, 0, 2, dbuf, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_predict(buf, 4, 2, None, dbuf, None) == sto.STO_EINVAL
    assert lib.sto_readout_nmse(buf, 4, 2, dbuf, dbuf, 0, 4, None, None) == sto.STO_EINVAL
    assert lib.sto_readout_nmse(buf, 4, 2, dbuf, dbuf, 2, 1, ctypes.byref(out), None) == sto.STO_EINVAL
    # row shards: the block must lie inside [0, N)
    cp = sto.Params().to_c()
    h = ctypes.c_void_p()
    for N, row0, rows in ((0, 0, 1), (8, -1, 2), (8, 0, 0), (8, 6, 3)):
        assert lib.sto_shard_create(N, row0, rows, ctypes.byref(cp), buf, buf, None, None,
                                    ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_shard_create(8, 0, 8, ctypes.byref(cp), None, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_shard_create(8, 0, 8, ctypes.byref(cp), buf, buf, None, None, None) == sto.STO_EINVAL
    bad = sto.Params(substeps=0).to_c()
    assert lib.sto_shard_create(8, 0, 8, ctypes.byref(bad), buf, buf, None, None, ctypes.byref(h)) == sto.STO_EINVAL
    assert lib.sto_shard_stage(None, buf, 0, None, 0, buf, None) == sto.STO_EINVAL
    assert lib.sto_shard_publish(None, buf) == sto.STO_EINVAL
    assert lib.sto_shard_get_state_f64(None, dbuf) == sto.STO_EINVAL
    lib.sto_shard_destroy(None)
    # groups and the single-launch sweep
    g = ctypes.c_void_p()
    assert lib.sto_group_create_ex(None, 1, 0, 0, ctypes.byref(g)) == sto.STO_EINVAL
    hs = (ctypes.c_void_p * 1)(None)
    assert lib.sto_group_create_ex(hs, 1, 0, -1, ctypes.byref(g)) == sto.STO_EINVAL
    assert lib.sto_run_sweep_group(None, None, buf, 1, None, None) == sto.STO_EINVAL
    assert lib.sto_batch_set_plan_threads(None, 40, 3, 1, 0, 512) == sto.STO_EINVAL
