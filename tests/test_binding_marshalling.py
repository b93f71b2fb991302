"""The Python binding without a GPU: argument marshalling and its checks.

A fake library records the C calls, and fake CUDA tensors stand in for
device buffers (the binding reads only their device, dtype, size,
contiguity and address). Each call must reach the library with the
pointers and sizes it was given. A field, gradient or workspace on another
device, a host or non-byte workspace, or a call made while another CUDA
device is current must be refused before any C call is made.
"""
import pytest
import torch

from paper_1101_0086_gb300 import mpa
from paper_1101_0086_gb300.workloads import dm_map


class FakeCuda:
    """Stands in for a contiguous CUDA tensor."""
    _next = 1 << 20

    def __init__(self, n, dtype, index=0, is_cuda=True, contiguous=True):
        self._n, self.dtype, self.is_cuda, self._c = int(n), dtype, is_cuda, contiguous
        self.device = torch.device("cuda", index) if is_cuda else torch.device("cpu")
        FakeCuda._next += 1 << 20
        self._ptr = FakeCuda._next

    def numel(self):
        return self._n

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return self._ptr


class FakeLib:
    """Records every C call; size queries answer fixed sizes."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def fn(*args):
            self.calls.append((name, args))
            out = {"mpa_plan_create": 1, "mpa_batch_create": 1}
            if name in out:
                args[-1]._obj.value = 0x1000
            elif name in ("mpa_plan_workspace_size", "mpa_batch_workspace_size", "ss_workspace_size",
                          "mpa_adjoint_workspace_size", "ss_adjoint_workspace_size"):
                args[-1]._obj.value = 4096
            elif name == "mpa_plan_n_segments":
                args[-1]._obj.value = 8
            return 0
        return fn


@pytest.fixture
def fake(monkeypatch):
    L = FakeLib()
    dev = {"cur": 0}
    real_empty, real_empty_like = torch.empty, torch.empty_like

    def empty(*size, dtype=None, device=None, **kw):
        d = torch.device(device) if device is not None else torch.device("cpu")
        if d.type == "cuda":
            n = size[0] if size and not isinstance(size[0], (tuple, list)) else size[0][0]
            return FakeCuda(n, dtype, d.index if d.index is not None else dev["cur"])
        return real_empty(*size, dtype=dtype, device=device, **kw)

    def empty_like(t, **kw):
        if isinstance(t, FakeCuda):
            return FakeCuda(t.numel(), t.dtype, t.device.index)
        return real_empty_like(t, **kw)

    monkeypatch.setattr(mpa, "lib", lambda: L)
    monkeypatch.setattr(torch, "empty", empty)
    monkeypatch.setattr(torch, "empty_like", empty_like)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: dev["cur"])
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: type("S", (), {"cuda_stream": 0})())
    L.dev = dev
    return L


N = 1 << 10


def make_plan(precision="fp32", **kw):
    return mpa.Plan(dm_map(4), N, 800.0, 5.0, 10, 2, precision=precision, **kw)


def test_plan_calls_reach_the_library_with_their_buffers(fake):
    plan = make_plan()
    assert plan.device == torch.device("cuda", 0) and plan.workspace.numel() == 4096
    f = FakeCuda(N, torch.complex64)
    plan.propagate(f, 0.0, 50.0)
    name, args = fake.calls[-1]
    assert name == "mpa_propagate" and args[1].value == f.data_ptr() and args[2:4] == (0.0, 50.0)
    psi0 = FakeCuda(N, torch.complex128)
    plan.interval(psi0, 5.0)
    assert fake.calls[-1][0] == "mpa_interval" and fake.calls[-1][1][1].value == psi0.data_ptr()
    ws = plan.propagate_checkpointed(f, 0.0, 50.0)
    name, args = fake.calls[-1]
    assert name == "mpa_propagate_checkpointed" and args[4].value == ws.data_ptr() and args[5] == ws.numel()
    g = FakeCuda(N, torch.complex64)
    gi, gs, gb = plan.adjoint(g, 0.0, 50.0, adj_workspace=ws)
    name, args = fake.calls[-1]
    assert name == "mpa_adjoint" and args[1] is None and args[2].value == g.data_ptr()
    assert args[6].value == ws.data_ptr() and gs.shape == (8,) and gb.shape == (8,)
    plan.autotune()
    assert fake.calls[-1][0] == "mpa_plan_autotune"


def test_module_level_forms(fake):
    plan = make_plan()
    f = FakeCuda(N, torch.complex64)
    assert mpa.propagate(f, plan, 0.0, 5.0) is f and fake.calls[-1][0] == "mpa_propagate"
    x = FakeCuda(N, torch.complex128)
    assert mpa.ss(x, dm_map(4), 800.0, 0.05, 0.0, 1.0) is x and fake.calls[-1][0] == "ss_propagate"


def test_plan_refuses_buffers_of_another_device_or_kind(fake):
    plan = make_plan()
    n_calls = len(fake.calls)
    with pytest.raises(ValueError, match="cuda:1"):
        plan.propagate(FakeCuda(N, torch.complex64, index=1), 0.0, 50.0)
    with pytest.raises(ValueError):
        plan.propagate(FakeCuda(N, torch.complex128), 0.0, 50.0)       # wrong precision
    with pytest.raises(ValueError):
        plan.propagate(FakeCuda(N, torch.complex64, contiguous=False), 0.0, 50.0)
    with pytest.raises(ValueError, match="workspace"):
        plan.adjoint(FakeCuda(N, torch.complex64), 0.0, 50.0, adj_workspace=FakeCuda(64, torch.float32))
    with pytest.raises(ValueError, match="workspace"):
        plan.adjoint(FakeCuda(N, torch.complex64), 0.0, 50.0, adj_workspace=FakeCuda(64, torch.uint8, index=1))
    fake.dev["cur"] = 1  # the plan's buffers are on cuda:0
    with pytest.raises(ValueError, match="current CUDA device"):
        plan.propagate(FakeCuda(N, torch.complex64), 0.0, 50.0)
    with pytest.raises(ValueError, match="current CUDA device"):
        plan.autotune()
    assert len(fake.calls) == n_calls  # nothing reached the library
    with pytest.raises(ValueError, match="workspace"):
        make_plan(workspace=FakeCuda(4096, torch.uint8, is_cuda=False))
    with pytest.raises(ValueError, match="workspace"):
        make_plan(workspace=FakeCuda(1024, torch.float32))


def test_plan_on_a_second_device_follows_its_workspace(fake):
    fake.dev["cur"] = 1
    plan = make_plan()                                   # "cuda" = the current device
    assert plan.device == torch.device("cuda", 1)
    plan.propagate(FakeCuda(N, torch.complex64, index=1), 0.0, 50.0)
    assert fake.calls[-1][0] == "mpa_propagate"
    with pytest.raises(ValueError):
        plan.propagate(FakeCuda(N, torch.complex64, index=0), 0.0, 50.0)


def test_batch_and_free_functions(fake):
    fields = [FakeCuda(N, torch.complex64), FakeCuda(2 * N, torch.complex64)]
    b = mpa.Batch([(dm_map(4), 800.0, 200.0, fields[0]), (dm_map(4), 1600.0, 100.0, fields[1])], 5.0, 10, 2)
    name, args = [c for c in fake.calls if c[0] == "mpa_batch_create"][-1]
    links = args[0]
    assert args[1] == 2 and [links[i].field for i in range(2)] == [f.data_ptr() for f in fields]
    b.propagate()
    assert fake.calls[-1][0] == "mpa_batch_propagate"
    with pytest.raises(ValueError):
        mpa.Batch([(dm_map(4), 800.0, 200.0, FakeCuda(N, torch.complex64, index=1))], 5.0, 10, 2)
    x = FakeCuda(N, torch.complex128)
    mpa.ss_propagate(x, dm_map(4), 800.0, 0.05, 0.0, 1.0)
    name, args = fake.calls[-1]
    assert name == "ss_propagate" and args[5].value == x.data_ptr() and args[9] == 4096
    mpa.fft(x, 1)
    assert fake.calls[-1][0] == "mpa_fft" and fake.calls[-1][1][3].value == x.data_ptr()
    mpa.fft_noalloc(x, -1)
    assert fake.calls[-1][0] == "mpa_fft_noalloc"
    gi, gs, gb = mpa.ss_adjoint(x, FakeCuda(N, torch.complex128), dm_map(4), 800.0, 0.05, 0.0, 1.0)
    assert fake.calls[-1][0] == "ss_adjoint" and gs.shape == (8,)
    with pytest.raises(ValueError):
        mpa.ss_adjoint(x, FakeCuda(N, torch.complex128, index=1), dm_map(4), 800.0, 0.05, 0.0, 1.0)
    with pytest.raises(ValueError, match="workspace"):
        mpa.ss_propagate(x, dm_map(4), 800.0, 0.05, 0.0, 1.0, workspace=FakeCuda(4096, torch.uint8, index=1))
    fake.dev["cur"] = 1
    with pytest.raises(ValueError, match="current CUDA device"):
        mpa.fft(x, 1)
    with pytest.raises(ValueError, match="current CUDA device"):
        b.propagate()
