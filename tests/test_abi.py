"""The C-ABI library builds, loads and exports every declared symbol; host-side
argument checks return error codes without touching a GPU."""
import ctypes

import pytest

from paper_2010_14258_gb300 import _lib, build


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(L):
    names = _lib.declared_symbols()
    assert "ldbp_apply" in names
    for name in names:
        assert hasattr(L, name), name


def test_version(L):
    assert L.ldbp_version() >= 100


def _apply(L, **kw):
    args = dict(taps=ctypes.c_void_p(16), stride=2, T=[3], c=[-0.1], M=1, x=ctypes.c_void_p(4096),
                y=ctypes.c_void_p(1 << 20), n=128, B=1, ckpt=None)
    args.update(kw)
    return L.ldbp_apply(args["taps"], args["stride"], _lib.i32_array(args["T"]) if args["T"] is not None else None,
                        _lib.f32_array(args["c"]) if args["c"] is not None else None, args["M"], args["x"],
                        args["y"], args["n"], args["B"], args["ckpt"], None)


@pytest.mark.parametrize("kw, needle", [
    (dict(x=None), "non-NULL"),
    (dict(taps=None), "non-NULL"),
    (dict(T=[4]), "odd"),
    (dict(T=[0]), "odd"),
    (dict(T=[35], stride=20), "supported length"),
    (dict(T=[7], stride=2), "taps_stride"),
    (dict(M=0, T=[3]), "M=0"),
    (dict(M=65, T=[3] * 65, c=[0.0] * 65), "M=65"),
    (dict(n=0), "n=0"),
    (dict(B=0), "batch=0"),
    (dict(y=ctypes.c_void_p(4096 + 8)), "overlap"),
    (dict(ckpt=ctypes.c_void_p(4096 + 512)), "ckpt overlaps"),
])
def test_ldbp_apply_rejects(L, kw, needle):
    rc = _apply(L, **kw)
    assert rc == -1
    assert needle in L.ldbp_last_error().decode()


def _apply_host(L, **kw):
    args = dict(x=ctypes.c_void_p(4096), y=ctypes.c_void_p(1 << 22), n=128, B=4, chunks=2,
                ws=ctypes.c_void_p(1 << 24), wsb=2 * 128 * 4 * 8)
    args.update(kw)
    return L.ldbp_apply_host(ctypes.c_void_p(16), 2, _lib.i32_array([3]), _lib.f32_array([-0.1]), 1, args["x"],
                             args["y"], args["n"], args["B"], args["chunks"], args["ws"], args["wsb"], None)


def test_apply_host_workspace_size(L):
    assert L.ldbp_apply_host_workspace(128, 4) == 2 * 128 * 4 * 8
    assert L.ldbp_apply_host_workspace(0, 4) == 0


@pytest.mark.parametrize("kw, needle", [
    (dict(x=None), "non-NULL"),
    (dict(chunks=0), "chunks=0"),
    (dict(chunks=5), "chunks=5"),
    (dict(wsb=100), "workspace"),
    (dict(ws=ctypes.c_void_p((1 << 24) + 8)), "aligned"),
    (dict(y=ctypes.c_void_p(4096 + 64)), "overlap"),
])
def test_ldbp_apply_host_rejects(L, kw, needle):
    assert _apply_host(L, **kw) == -1
    assert needle in L.ldbp_last_error().decode()


@pytest.mark.parametrize("v", [float("nan"), float("inf")])
def test_ldbp_apply_rejects_nonfinite_coefficient(L, v):
    assert _apply(L, c=[v]) == -6
    assert "NaN or infinite" in L.ldbp_last_error().decode()


def _essm(L, kappa=(2,), stride=5, eta=ctypes.c_void_p(64), T=(3,)):
    M = len(T)
    return L.ldbp_essm_apply(ctypes.c_void_p(16), 2, _lib.i32_array(list(T)), _lib.f32_array([-0.1] * M), eta, stride,
                             _lib.i32_array(list(kappa)), M, ctypes.c_void_p(4096), ctypes.c_void_p(1 << 20), 128, 1,
                             None, None)


@pytest.mark.parametrize("kw, needle", [
    (dict(eta=None), "non-NULL"),
    (dict(kappa=(25,), stride=51), "kappa[0]=25"),
    (dict(kappa=(3,), stride=5), "eta_stride"),
    (dict(T=(19,)), "supported length"),
])
def test_ldbp_essm_apply_rejects(L, kw, needle):
    assert _essm(L, **kw) == -1
    assert needle in L.ldbp_last_error().decode()


def _resample(L, **kw):
    args = dict(x=ctypes.c_void_p(4096), n_in=1536, y=ctypes.c_void_p(1 << 22), n_out=512, bw=1.0, B=2)
    args.update(kw)
    return L.ldbp_resample(args["x"], args["n_in"], args["y"], args["n_out"], args["bw"], args["B"], None)


@pytest.mark.parametrize("kw, needle", [
    (dict(x=None), "non-NULL"),
    (dict(bw=0.0), "bandwidth"),
    (dict(bw=1.5), "bandwidth"),
    (dict(n_out=500), "divide"),
    (dict(n_in=999, n_out=333), "power of two"),       # odd coarse grid
    (dict(n_in=768, n_out=256), "power of two"),        # coarse grid below 512
    (dict(n_in=9 * 512, n_out=512), "ratio"),           # r = 9
    (dict(n_in=8 * 4096, n_out=4096), "at most 16384"),  # fine grid too long
    (dict(B=0), "batch=0"),
    (dict(x=ctypes.c_void_p(4096 + 8)), "aligned"),
    (dict(y=ctypes.c_void_p(4096 + 64)), "overlap"),
])
def test_resample_rejects(L, kw, needle):
    assert _resample(L, **kw) == -1
    assert needle in L.ldbp_last_error().decode()


def test_resample_rejects_nonfinite_bandwidth(L):
    assert _resample(L, bw=float("nan")) == -6


def _split_step(L, fn, n, **kw):
    import synth
    from paper_2010_14258_gb300 import api
    f = api.fiber_struct(synth.Fiber(**kw.pop("fiber", {})))
    lk = api.link_struct(synth.Link(**kw.pop("link", {})))
    x, y = ctypes.c_void_p(4096), ctypes.c_void_p(1 << 22)
    if fn == "ssm_forward":
        return L.ssm_forward(ctypes.byref(f), ctypes.byref(lk), 20e9, x, y, n, 1, None)
    return L.ssm_cufft(ctypes.byref(f), ctypes.byref(lk), 20e9, 0, 0, x, y, n, 1, None)


@pytest.mark.parametrize("fn, n, needle", [
    ("ssm_forward", 5120, "power of two"),   # the fused kernel takes 2^k and 3 * 2^k only
    ("ssm_forward", 256, "power of two"),
    ("ssm_forward", 768, "three times"),     # 3 * 2^8: below the 3 * 2^k range
    ("ssm_forward", 3 << 15, "three times"),  # above it
    ("ssm_cufft", 1, "[2, 2^27]"),          # the library-FFT path takes any length
    ("ssm_cufft", (1 << 27) + 1, "[2, 2^27]"),
])
def test_split_step_length_checks(L, fn, n, needle):
    assert _split_step(L, fn, n) == -1
    assert needle in L.ldbp_last_error().decode()


@pytest.mark.parametrize("kw, code, needle", [
    (dict(link=dict(n_spans=0)), -1, "n_spans >= 1"),
    (dict(fiber=dict(alpha_db_per_km=-0.1)), -1, "alpha"),
    (dict(fiber=dict(gamma_per_w_km=float("nan"))), -6, "NaN"),
])
def test_split_step_parameter_checks(L, kw, code, needle):
    for fn in ("ssm_forward", "ssm_cufft"):
        assert _split_step(L, fn, 4096, **dict(kw)) == code
        assert needle in L.ldbp_last_error().decode()


def test_wait_probe_rejects_bad_arguments(L):
    # host-side checks: nothing is launched
    assert L.ldbp_wait_probe(3, 10, None) == -1
    assert L.ldbp_wait_probe(-1, 10, None) == -1
    assert L.ldbp_wait_probe(1, 0, None) == -1
    assert L.ldbp_wait_probe(1, (1 << 20) + 1, None) == -1
    assert b"limit" in L.ldbp_last_error()


def test_ragged_set_schedule_rejects_null_plan(L):
    assert L.ldbp_ragged_set_schedule(None, 2048, 1) == -1
    assert b"plan" in L.ldbp_last_error()
