"""The fixed-footprint statistics entry point (tf_phi_stats_noalloc).

It serves callers that cannot hand the library device memory at call time:
it must give the same concentration mean and standard deviation as the
workspace-based tf_phi_stats while allocating nothing, and it keeps its
partial sums in one statically allocated device array shared by all calls.
This file is named to be collected last; it passes alone in a fresh process
and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from paper_2511_00445_gb300 import _binding as B

pytestmark = pytest.mark.gpu


def _call(lib, values, n, ref, out, stream):
    return lib.tf_phi_stats_noalloc(ctypes.c_void_p(values.data_ptr()), n, ref,
                                    ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_stats_match_workspace_entry_point_on_two_calls():
    import torch

    from paper_2511_00445_gb300 import build
    build.build()
    lib = B.load_library()
    p = B.SolverParams(nx=160, ny=96, zeta=0.01)
    tf = B.TwoFluid(p)
    tf.init_fields(seed=21, phi0=0.5, dphi=0.05, S0=0.2)
    stream = tf.stream
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for call in range(2):
        if call == 1:
            tf.step(15)   # a different field for the second call
        mean_ref, std_ref = tf.phi_stats(0)
        phi = tf.read_field(0, B.FIELD_PHI)
        # the stored deviations phi - phi_ref, exactly
        dev = torch.tensor((phi - 0.5).astype(np.float32).ravel(), device="cuda")
        out.fill_(float("nan"))
        assert _call(lib, dev, dev.numel(), 0.5, out, stream) == B.TF_OK
        stream.synchronize()
        m, s = out.tolist()
        assert abs(m - mean_ref) < 1e-12
        assert abs(s - std_ref) < 1e-9 * std_ref
    tf.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2511_00445_gb300 import build
    build.build()
    lib = B.load_library()
    stream = torch.cuda.current_stream()
    dev = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _call(lib, dev, B.NOALLOC_MAX_ELEMS + 1, 0.0, out, stream) == B.TF_ERR_TOO_LARGE
    assert _call(lib, dev, 0, 0.0, out, stream) == B.TF_ERR_ARG
    assert lib.tf_phi_stats_noalloc(None, 8, 0.0, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream)) == B.TF_ERR_ARG


def _host_stats(v32):
    v = v32.astype(np.float64)
    m = v.mean()
    return m, float(np.sqrt(np.mean((v - m) ** 2)))


def test_noalloc_at_its_size_limit_and_after_larger_calls():
    """n = TF_NOALLOC_MAX_ELEMS (every partial slot) and MAX - 1 (a ragged last
    block), each preceded and followed by small calls: every result matches an
    FP64 two-pass host computation of the same FP32 values, so no partial left
    by an earlier, larger call leaks into a later one.  The large inputs are
    not centred (mean 300, spread ~1e-2)."""
    import torch

    from paper_2511_00445_gb300 import build
    build.build()
    lib = B.load_library()
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(7)
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    small = (0.01 * rng.standard_normal(5000)).astype(np.float32)
    big = (300.0 + 0.01 * rng.standard_normal(B.NOALLOC_MAX_ELEMS)).astype(np.float32)
    cases = [small, big, small[:4097], big[:-1], small[:1], small]
    for v in cases:
        dev = torch.tensor(v, device="cuda")
        out.fill_(float("nan"))
        assert _call(lib, dev, dev.numel(), 0.25, out, stream) == B.TF_OK
        stream.synchronize()
        m, s = out.tolist()
        hm, hs = _host_stats(v)
        assert abs(m - (0.25 + hm)) <= 1e-12 * max(1.0, abs(hm)), (v.size, m, hm)
        assert abs(s - hs) <= 1e-9 * hs + 1e-300, (v.size, s, hs)
