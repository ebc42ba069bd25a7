"""Host logic of the Python binding's contact_step_host wrapper (no GPU: a
fake library records the arguments): the checked arguments are reused only
when the caller passes the same tensor objects with the same storage, never
for calls that allocate outputs or ask for the pair outputs; a rejected call
raises and leaves nothing cached."""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_2401_10878_gb300 import contact as C  # noqa: E402


class FakeLib:
    def __init__(self):
        self.calls = []
        self.rc = 0

    def contact_step_host(self, ctx, *args):
        self.calls.append(tuple(a.value if isinstance(a, ctypes.c_void_p) else a for a in args))
        return self.rc

    def contact_last_error(self, ctx):
        return b"fake"


def model(n=5):
    m = C.Contact.__new__(C.Contact)
    m.n, m.max_pairs, m.steps, m.ctx = n, 16, 0, None
    m.lib = FakeLib()
    return m


def tensors(n=5):
    return (torch.zeros((n, 3), dtype=torch.float64), torch.zeros((n, 4), dtype=torch.float64),
            torch.zeros((n, 3), dtype=torch.float64), torch.zeros((n, 3), dtype=torch.float64))


def test_same_buffers_reuse_the_checked_arguments():
    m = model()
    p, q, f, t = tensors()
    m.step_host(p, q, force=f, torque=t)
    assert m._host_fast is not None
    m.step_host(p, q, force=f, torque=t)
    a, b = m.lib.calls
    assert a == b and a[0] == p.data_ptr() and a[4] == f.data_ptr() and m.steps == 2


def test_new_objects_or_storage_take_the_checked_path():
    m = model()
    p, q, f, t = tensors()
    m.step_host(p, q, force=f, torque=t)
    p2 = p.clone()
    m.step_host(p2, q, force=f, torque=t)
    assert m.lib.calls[-1][0] == p2.data_ptr()
    p2.set_(torch.zeros((5, 3), dtype=torch.float64))   # same object, new storage
    m.step_host(p2, q, force=f, torque=t)
    assert m.lib.calls[-1][0] == p2.data_ptr()


def test_allocated_outputs_and_pairs_are_never_cached():
    m = model()
    p, q, f, t = tensors()
    m.step_host(p, q)                       # outputs allocated by the wrapper
    assert m._host_fast is None
    m.step_host(p, q, force=f, torque=t, pairs=True)
    assert m._host_fast is None
    out = m.step_host(p, q, force=f, torque=t, pairs=True)
    assert "pair_out" in out


def test_bad_shapes_are_refused_and_errors_raise():
    m = model()
    p, q, f, t = tensors()
    with pytest.raises(C.ContactError):
        m.step_host(torch.zeros((4, 3), dtype=torch.float64), q, force=f, torque=t)
    m.lib.rc = C.EINVAL
    with pytest.raises(C.ContactError):
        m.step_host(p, q, force=f, torque=t)
