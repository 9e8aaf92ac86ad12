"""The allocation-free entry point ss_run_noalloc against the context API.

ss_run_noalloc serves callers that cannot call cudaMalloc: a host that owns
all device memory through its own pool, a framework with a device memory
budget fixed at start-up, real-time loops in which an allocation could block.
Its kernel scratch lives in one file-scope device array; the caller passes the
state and the outputs.  This test drives it through the C ABI on caller-owned
device buffers and checks two calls in a row against ss_run on a context
started from the same state: integers equal, positions within the parity
tolerances (1e-10 in FP64, 1e-4 relative in FP32), correlator sums of each
call within 1e-9 relative.  One case runs under simple shear (the velocity
gradient set from step 0 on the context, passed to each allocation-free call).
The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_1106_2899_gb300 import SlipSpring
from paper_1106_2899_gb300 import _native as nat

pytestmark = pytest.mark.gpu


def _lanes(N):
    """NP, the padded bead/slot count of the device layout."""
    return -(-N // 16) * 16 if N <= 64 else 128


def _to_device_layout(st, N, zm, dtype):
    M = st["R"].shape[0]
    W = _lanes(N)
    R = np.zeros((M, 3, W), dtype=dtype)
    A = np.zeros((M, 3, W), dtype=dtype)
    S = -np.ones((M, W), dtype=np.int32)
    R[:, :, :N] = np.transpose(st["R"], (0, 2, 1)).astype(dtype)
    for m in range(M):
        z = int(st["Z"][m])
        S[m, :z] = st["S"][m, :z]
        A[m, :, :z] = st["A"][m, :z].T.astype(dtype)
    return R, A, S, np.ascontiguousarray(st["Z"], dtype=np.int32)


def _from_device_layout(R, A, S, Z, N, zm):
    M = R.shape[0]
    out = {"R": np.transpose(R[:, :, :N], (0, 2, 1)).astype(np.float64), "Z": Z.copy(),
           "S": -np.ones((M, zm), dtype=np.int32), "A": np.zeros((M, zm, 3))}
    for m in range(M):
        z = int(Z[m])
        out["S"][m, :z] = S[m, :z]
        out["A"][m, :z] = A[m, :, :z].T
    return out


def _noalloc_call(lib, params, precision, seed, M, N, t0, n, dev, corr, status, stream, kappa=None):
    R, A, S, Z = dev
    kap = None
    if kappa is not None:
        # a fresh host array per call, released right after it: the call must
        # not keep reading it
        kap = np.ascontiguousarray(kappa, dtype=np.float64).reshape(9).copy()
    rc = lib.ss_run_noalloc(C.byref(params), precision, seed, M, N, 0, t0, n,
                            kap.ctypes.data_as(C.POINTER(C.c_double)) if kap is not None else None,
                            C.c_void_p(R.data_ptr()),
                            C.c_void_p(A.data_ptr()), C.c_void_p(S.data_ptr()), C.c_void_p(Z.data_ptr()),
                            C.c_void_p(corr.data_ptr()), C.c_void_p(status.data_ptr()), C.c_void_p(stream))
    assert rc == 0, nat.ERRORS.get(rc, rc)


@pytest.mark.parametrize("precision,N,gdot", [("fp64", 16, 0.0), ("fp32", 32, 0.0), ("fp32", 80, 0.0),
                                             ("fp32", 32, 0.05), ("fp64", 24, 0.05)])
def test_noalloc_two_calls_match_context(cuda_ok, precision, N, gdot):
    import torch

    from paper_1106_2899_gb300 import build
    build.build()
    lib = nat.load()
    M, seed, levels, n1, n2 = 200, 11, 10, 300, 500
    zm = min(N, 64)
    st0 = synth.random_state(M, N, zm, seed=3, z_mean=N / 4)
    kw = dict(corr_levels=levels, groups=4, chunk_steps=128)
    prec = nat.SS_FP64 if precision == "fp64" else nat.SS_FP32
    dtype = np.float64 if precision == "fp64" else np.float32

    # the existing entry points, on a context
    kappa = synth.shear_kappa(gdot) if gdot else None
    g = SlipSpring([(M, N)], precision=precision, seed=seed)
    g.set_params(**kw)
    g.set_state(st0)
    if kappa is not None:
        g.set_flow(kappa, from_step=0)
    g.run(n1)
    ref1, acc1 = g.get_state(), g.corr_sums()[0].sum(axis=0)
    g.reset_observables()
    g.run(n2)
    ref2, acc2 = g.get_state(), g.corr_sums()[0].sum(axis=0)
    g.close()

    # the allocation-free entry point on caller-owned device buffers
    params = nat.ss_params()
    for k, v in kw.items():
        setattr(params, k, v)
    dev = [torch.from_numpy(x).cuda() for x in _to_device_layout(st0, N, zm, dtype)]
    corr = torch.zeros((levels, 16, 2, 3), dtype=torch.float64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lags = np.array([[(k << l) if (l == 0 or k >= 8) else -1 for k in range(16)] for l in range(levels)])
    rtol = 1e-10 if precision == "fp64" else 1e-4
    for call, (t0, n, ref, acc) in enumerate([(0, n1, ref1, acc1), (n1, n2, ref2, acc2)]):
        _noalloc_call(lib, params, prec, seed, M, N, t0, n, dev, corr, status, stream, kappa)
        torch.cuda.synchronize()
        got = _from_device_layout(*[x.cpu().numpy() for x in dev], N, zm)
        assert int(status.item()) == 0
        assert np.array_equal(got["Z"], ref["Z"]), "call %d: Z" % call
        assert np.array_equal(got["S"], ref["S"]), "call %d: S" % call
        assert np.all(np.abs(got["R"] - ref["R"]) <= rtol * np.maximum(1, np.abs(ref["R"]))), "call %d: R" % call
        assert np.all(np.abs(got["A"] - ref["A"]) <= rtol * np.maximum(1, np.abs(ref["A"]))), "call %d: A" % call
        co = corr.cpu().numpy()
        used = lags >= 0
        scale = np.abs(acc[used]).max()
        assert np.allclose(co[used], acc[used], rtol=1e-9, atol=1e-12 * scale), "call %d: correlator" % call


def test_noalloc_rejects_oversized_request(cuda_ok):
    lib = nat.load()
    params = nat.ss_params()
    params.corr_levels = 24
    # scratch grows with chains x levels: far beyond 32 MiB, refused before any launch
    rc = lib.ss_run_noalloc(C.byref(params), nat.SS_FP32, 0, 1 << 20, 32, 0, 0, 1, None, C.c_void_p(1),
                            C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), None, None, None)
    assert rc == -7
    params.log_every = 10
    rc = lib.ss_run_noalloc(C.byref(params), nat.SS_FP32, 0, 8, 32, 0, 0, 1, None, C.c_void_p(1),
                            C.c_void_p(1), C.c_void_p(1), C.c_void_p(1), None, None, None)
    assert rc == -1
