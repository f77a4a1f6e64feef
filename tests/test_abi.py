"""The C-ABI library loads and exports every entry point its header
declares (no compute calls: this runs without a GPU)."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mlmc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1904_12754_gb300 import mlmc
    return mlmc.load()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("mlmc_plan_create", "mlmc_expmv", "mlmc_stats", "mlmc_plan_destroy",
                 "mlmc_last_error", "mlmc_mlmcl", "mlmc_trace"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_1904_12754_gb300 import mlmc
    s = mlmc.schedule_default()
    assert s.l0 == -1 and s.num_levels == 5 and s.precision == mlmc.FP64
    assert lib.mlmc_plan_create(None, 1, 0, None, None, None, 0.0, None, 1e-3, None) == \
        mlmc.MLMC_ERR_INVALID_ARG
    assert b"NULL" in lib.mlmc_last_error()
    h = ct.c_void_p()
    # rejected before any device work: negative t, bad tolerance, n = 0
    rp = (ct.c_int64 * 2)(0, 0)
    for n, t, tol in ((1, -1.0, 1e-3), (1, 1.0, 0.0), (0, 1.0, 1e-3)):
        st = lib.mlmc_plan_create(ct.byref(h), n, 0, rp, None, None, t, None, tol, None)
        assert st == mlmc.MLMC_ERR_INVALID_ARG
    lib.mlmc_plan_destroy(None)


def test_schedule_checks_come_before_device_work(lib):
    # Every bad schedule is refused with INVALID_ARG and a message, before the
    # plan touches the device (this runs without a GPU).
    from paper_1904_12754_gb300 import mlmc
    rp = (ct.c_int64 * 2)(0, 0)
    h = ct.c_void_p()

    def create(**fields):
        s = mlmc.schedule_default()
        for k, v in fields.items():
            setattr(s, k, v)
        return lib.mlmc_plan_create(ct.byref(h), 1, 0, rp, None, None, 1.0, ct.byref(s), 1e-3, None)

    bad = [dict(num_levels=0), dict(num_levels=4, max_levels=3), dict(max_levels=33),
           dict(precision=7), dict(mode=5), dict(proposal=1), dict(pilot_walks=1),
           dict(max_walks_per_row=1), dict(max_jumps_per_walk=-1), dict(l0=25),
           dict(l0=20, num_levels=3, max_levels=6), dict(l2_persist=2),
           dict(block_threads=48), dict(block_threads=512), dict(walks_per_lane=-1),
           dict(launch_reps=-1)]
    for fields in bad:
        assert create(**fields) == mlmc.MLMC_ERR_INVALID_ARG, fields
        assert lib.mlmc_last_error(), fields
        assert not h.value


def test_every_entry_point_refuses_null_handles(lib):
    # Each status-returning call of the header, given NULL handles and zero
    # sizes, returns INVALID_ARG with a message and does no device work.
    from paper_1904_12754_gb300 import mlmc
    skip = {"mlmc_last_error", "mlmc_launch_count", "mlmc_plan_destroy", "mlmc_batch_destroy",
            "mlmc_mlp_destroy", "mlmc_plan_tilt_pieces"}
    assert lib.mlmc_plan_tilt_pieces(None) == 0     # a count, not a status: 0 for no plan
    called = 0
    for name in _declared():
        fn = getattr(lib, name)
        if name in skip or fn.argtypes is None or fn.restype not in (ct.c_int, ct.c_int32):
            continue
        args = []
        for t in fn.argtypes:
            if t in (ct.c_double, ct.c_float):
                args.append(t(0.0))
            elif isinstance(t, type) and issubclass(t, (ct.c_int, ct.c_int32, ct.c_int64, ct.c_uint32,
                                                        ct.c_uint64, ct.c_bool)):
                args.append(t(0))
            else:
                args.append(None)
        assert fn(*args) == mlmc.MLMC_ERR_INVALID_ARG, name
        assert lib.mlmc_last_error(), name
        called += 1
    assert called >= 20
