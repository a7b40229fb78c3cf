"""The binding refuses wrongly sized, typed or placed vectors before any
library call, and the library refuses overlapping input and output device
vectors before any device work (no GPU needed: the pointers are never
dereferenced)."""
import ctypes as C

import numpy as np
import pytest

from owqs_inputs.patterns import E, M, N, Pattern


@pytest.fixture(scope="module")
def owqs():
    from paper_1604_05659_gb300 import build, owqs as mod
    build.ensure_built()
    mod.library()
    return mod


class FakeTensor:
    """Stands in for a CUDA tensor: only the attributes the checks read."""

    def __init__(self, n, dtype="c64", cuda=True, contiguous=True, device="cuda:0"):
        self._n, self.dtype, self.is_cuda, self._c, self.device = n, dtype, cuda, contiguous, device

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c


def test_device_vector_checks(owqs):
    chk = owqs._check_vectors
    chk(FakeTensor(8), FakeTensor(4), "c64", 3, 2)                 # exact sizes
    chk(None, FakeTensor(5), "c64", 3, 2)                          # a larger out is allowed
    chk(FakeTensor(8), None, "c64", 3, 2)                          # the binding allocates out
    bad = [
        (FakeTensor(4), FakeTensor(4)),                            # psi_in short
        (FakeTensor(16), FakeTensor(4)),                           # psi_in long
        (FakeTensor(8), FakeTensor(3)),                            # out short
        (FakeTensor(8, dtype="c128"), FakeTensor(4)),              # psi_in dtype
        (FakeTensor(8), FakeTensor(4, dtype="c128")),              # out dtype
        (FakeTensor(8, cuda=False), FakeTensor(4)),                # host tensor as psi_in
        (FakeTensor(8), FakeTensor(4, cuda=False)),                # host tensor as out
        (FakeTensor(8, contiguous=False), FakeTensor(4)),
        (FakeTensor(8), FakeTensor(4, contiguous=False)),
        (FakeTensor(8), FakeTensor(4, device="cuda:1")),           # two devices
    ]
    for pin, out in bad:
        with pytest.raises(ValueError):
            chk(pin, out, "c64", 3, 2)
    with pytest.raises(ValueError):                                # a unitary writes 2^(|O| + |I|)
        chk(None, FakeTensor(16), "c64", 0, 5)


def test_host_vector_checks(owqs):
    chk = owqs._check_host_vectors
    chk(np.zeros(8, np.complex64), np.zeros(4, np.complex64), "c64", 3, 2)
    chk(None, np.zeros(4, np.complex128), "c128", 3, 2)
    for pin, out in [(np.zeros(4, np.complex64), np.zeros(4, np.complex64)),
                     (np.zeros(8, np.complex64), np.zeros(2, np.complex64)),
                     (np.zeros(8, np.complex128), np.zeros(4, np.complex64)),
                     (np.zeros(16, np.complex64)[::2], np.zeros(4, np.complex64)),
                     ([0j] * 8, np.zeros(4, np.complex64))]:
        with pytest.raises(ValueError):
            chk(pin, out, "c64", 3, 2)
    ro = np.zeros(4, np.complex64)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        chk(None, ro, "c64", 3, 2)
    torch = pytest.importorskip("torch")                           # CPU torch tensors (pinned in practice)
    chk(torch.zeros(8, dtype=torch.complex64), torch.zeros(4, dtype=torch.complex64), "c64", 3, 2)
    for pin, out in [(torch.zeros(8, dtype=torch.complex128), None),
                     (torch.zeros(16, dtype=torch.complex64)[::2], None),
                     (None, torch.zeros(2, dtype=torch.complex64))]:
        with pytest.raises(ValueError):
            chk(pin, out, "c64", 3, 2)


def _wires(owqs):
    # three input qubits, one measured: 8 input and 4 output amplitudes
    p = Pattern(4, [0, 1, 2], [1, 2, 3], [N(3), E(0, 3), M(0, 0.3)], "three wires")
    return owqs.load(p)


@pytest.mark.parametrize("entry", ["owqs_run", "owqs_run_static"])
def test_overlapping_device_vectors_are_refused_before_device_work(owqs, entry):
    h = _wires(owqs)
    fn = getattr(owqs.library(), entry)
    oc = (C.c_uint8 * 1)(0)
    for dtype, amp in (("c64", 8), ("c128", 16)):
        opts = owqs.owqs_run_opts(owqs.DTYPE[dtype], owqs.MODE["owqs"], owqs.POLICY["forced"], 0, 0, None, 0, 0)
        base = 1 << 20
        last = 8 * amp - 16                            # the input's last 16-byte-aligned offset
        for off in (0, 16, last):                      # the same start, or inside the other vector
            st = fn(h._h, C.byref(opts), C.c_void_p(base), C.c_void_p(base + off), oc, None)
            assert st == owqs.ERR_ARG and "overlap" in owqs.last_error(), (entry, dtype, off, st)
            if off < 4 * amp:                          # the output is 4 amplitudes long
                st = fn(h._h, C.byref(opts), C.c_void_p(base + off), C.c_void_p(base), oc, None)
                assert st == owqs.ERR_ARG and "overlap" in owqs.last_error(), (entry, dtype, off, st)
        # adjacent vectors pass this check (the call then fails on the missing device, or runs on a GPU
        # box: it is made only where there is no device)
        pytest.importorskip("torch")
        import torch
        if not torch.cuda.is_available():
            st = fn(h._h, C.byref(opts), C.c_void_p(base), C.c_void_p(base + 8 * amp), oc, None)
            assert "overlap" not in owqs.last_error()
