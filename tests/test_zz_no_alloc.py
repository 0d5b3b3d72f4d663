"""fs_apply_H_static: the FP64 H application that allocates no device memory.

Some callers cannot call cudaMalloc when they apply H (a restricted or
pre-planned allocator); this entry point keeps all of its intermediates in a
64 MiB array the library declares on the device.  The test calls it through
the C ABI twice in a row and compares both results with fs_apply_H (the same
operator with library-allocated buffers) at the FP64 parity tolerance, and
checks that a problem whose single band needs more scratch than the array is
rejected with a clear message.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import fs_inputs as fi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1907_06821_gb300 import build as b
    b.build()
    import paper_1907_06821_gb300 as m
    return m


def _cases():
    return {
        "tiny": fi.make_config("tiny"),
        "box_two_widths": fi.make_box(L=(12.0, 12.0, 12.0), n=(20, 24, 40), ecut=4.0, k=(0.0, 0.05, 0.0),
                                      natom=5, widths=(0.8, 1.2), nstates=10, e_ref=0.2, seed=8),
    }


@pytest.mark.parametrize("case", ["tiny", "box_two_widths"])
def test_static_scratch_matches_apply_H(fs, case):
    w = _cases()[case]
    with fs.Context.from_workload(w) as c:
        X = torch.from_numpy(fi.raw_start_block(21, c.npw, 31)).cuda()
        ref = c.apply_H(X, shift=0.17).cpu().numpy()
        scale = np.abs(ref).max()
        for _ in range(2):                       # two calls in a row share the static array
            out = torch.empty_like(X)
            st = c.lib.fs_apply_H_static(c.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         X.shape[0], ctypes.c_double(0.17))
            assert st == fs.FS_OK, c.lib.fs_last_error(c.h)
            assert np.abs(out.cpu().numpy() - ref).max() / scale < 1e-12


def test_static_scratch_several_chunks(fs):
    """The wire grid (72 x 72 x 144, 193,673 plane waves, 2,048 projectors) needs about
    6 MB of scratch per band, so 23 bands run in three chunks of the 64 MiB array
    (11, 11 and a ragged last chunk of 1): the chunk offsets and the reuse of the
    column buffer, projections and partial sums across chunks are exercised."""
    w = fi.make_config("wire")
    with fs.Context.from_workload(w) as c:
        X = torch.from_numpy(fi.raw_start_block(23, c.npw, 41)).cuda()
        ref = c.apply_H(X, shift=-0.05)
        scale = ref.abs().max().item()
        for _ in range(2):
            out = torch.empty_like(X)
            st = c.lib.fs_apply_H_static(c.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         X.shape[0], ctypes.c_double(-0.05))
            assert st == fs.FS_OK, c.lib.fs_last_error(c.h)
            assert (out - ref).abs().max().item() / scale < 1e-12


def test_static_scratch_rejects_oversized_band(fs):
    # 108 x 108 x 720 grid and a 20 Ha sphere: one band's column buffer alone is ~90 MB
    L, n = (50.0, 50.0, 100.0), (108, 108, 720)
    with fs.Context(L, n, 20.0, (0.0, 0.0, 0.0), np.zeros(n)) as c:
        X = torch.zeros((1, c.npw), dtype=torch.complex128, device="cuda")
        out = torch.empty_like(X)
        st = c.lib.fs_apply_H_static(c.h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1,
                                     ctypes.c_double(0.0))
        assert st == fs.FS_ERR_ARG
        assert b"bytes of scratch" in c.lib.fs_last_error(c.h)
