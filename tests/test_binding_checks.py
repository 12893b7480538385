"""The Python binding refuses buffers the C library would read or write past
the end of: wrong dtype, wrong shape, mismatched x / y, a shift list whose
length is not the batch size.  These checks run before any library call, so
they are tested here on CPU tensors with the operator and factor sizes
stubbed (no GPU, no handle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_01458_gb300 import _lib  # noqa: E402

N, B, Q, NX, NY = 60, 12, 3, 5, 4
FAKE_OP = 0x1000
FAKE_FA = 0x2000


@pytest.fixture
def stubbed(monkeypatch):
    monkeypatch.setattr(_lib, "rr_operator_dims", lambda h: (N, B, Q, NX, NY))
    monkeypatch.setitem(_lib._FA_DIMS, FAKE_FA, (2, N, 0, NX * NY))

    def no_library():
        raise AssertionError("the binding reached the library with a bad buffer")

    monkeypatch.setattr(_lib, "load", no_library)


def _c128(*shape):
    return torch.zeros(*shape, dtype=torch.complex128)


@pytest.mark.parametrize("fn", ["rr_apply", "rr_apply_static"])
def test_apply_rejects_bad_buffers(stubbed, fn):
    call = getattr(_lib, fn)
    shifts = np.array([0.5j, 1.0j])
    cases = [
        (torch.zeros(2, N, 3, dtype=torch.complex64), _c128(2, N, 3), "dtype"),
        (_c128(2, N, 3), torch.zeros(2, N, 3, dtype=torch.complex64), "dtype"),
        (_c128(2, N - 1, 3), _c128(2, N - 1, 3), "shape"),
        (_c128(2, N, 3), _c128(2, N, 2), "shape"),
        (_c128(3, N, 3), _c128(3, N, 3), "shape"),      # 3 problems, 2 shifts
        (_c128(N, 3), _c128(N, 3), "[F, N, k]"),
        (_c128(2, N, 3), _c128(2, N, 3), "CUDA"),       # right shape, host memory
    ]
    for x, y, what in cases:
        with pytest.raises(ValueError, match=what.replace("[", r"\[").replace("]", r"\]")):
            call(FAKE_OP, shifts, x, y)
    with pytest.raises(ValueError, match="shift"):
        call(FAKE_OP, np.array([], dtype=np.complex128), _c128(0, N, 1), _c128(0, N, 1))


def test_factor_calls_reject_bad_buffers(stubbed):
    good = _c128(2, N, 4)
    sig = torch.zeros(2, 4, dtype=torch.float64)
    with pytest.raises(ValueError, match="shape"):
        _lib.rr_solve(FAKE_FA, good, _c128(2, N, 5))
    with pytest.raises(ValueError, match="dtype"):
        _lib.rr_solve(FAKE_FA, good, torch.zeros(2, N, 4, dtype=torch.complex64))
    with pytest.raises(ValueError, match="shape"):
        _lib.rr_modes(FAKE_FA, 4, good, _c128(1, N, 4), sig)
    with pytest.raises(ValueError, match="shape"):
        _lib.rr_modes(FAKE_FA, 4, good, _c128(2, N, 4), torch.zeros(2, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="seeds"):
        _lib.rr_sketch(FAKE_FA, 4, [1, 2, 3], None, good, sig)
    with pytest.raises(ValueError, match="phi"):
        _lib.rr_sketch(FAKE_FA, 4, [1, 2], torch.zeros(N + 1, dtype=torch.float64), good, sig)
    with pytest.raises(ValueError, match="grad"):
        _lib.rr_gain_grad(FAKE_FA, 2, good, _c128(2, N, 4), sig,
                          torch.zeros(3 * NX * NY - 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="one shift per problem"):
        _lib.rr_refactor(FAKE_FA, [1j])
    with pytest.raises(ValueError, match="unknown factors handle"):
        _lib.rr_solve(0x3000, good, _c128(2, N, 4))


def test_test_matrix_rejects_bad_buffers(stubbed):
    with pytest.raises(ValueError, match="shape"):
        _lib.rr_gaussian([1, 2], N, 3, None, _c128(1, N, 3))
    with pytest.raises(ValueError, match="phi"):
        _lib.rr_test_matrix([1], N, 3, torch.zeros(N - 1, dtype=torch.float64),
                            _c128(1, N, 3), kind="rademacher")
