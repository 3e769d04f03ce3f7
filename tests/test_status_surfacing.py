"""Device errors reach the autograd caller (CPU, no GPU): the solver entry
points are replaced by host-side fakes whose context reports the status a
real launch would leave in the device status word -- RF_ERR_NOT_CONVERGED
when the forward is given max_sweeps = 1, RF_ERR_TIMEOUT from the adjoint --
and RFSolve / SweepSolve / the inverse driver must raise instead of returning
gradients of an unusable T."""
import pytest

torch = pytest.importorskip("torch")

from paper_2603_00035_gb300 import _lib as L  # noqa: E402
from paper_2603_00035_gb300 import api, autograd  # noqa: E402


class FakeCtx:
    def __init__(self):
        self.pending = L.RF_OK

    def stats(self):
        st, self.pending = self.pending, L.RF_OK  # read-and-clear, as rf_ctx_last_stats
        return dict(status=st, status_name=L.STATUS[st], sweeps=1, converged=st == L.RF_OK, adj_sweeps=0,
                    cell_updates=0, max_residual=0.0)

    raise_on_device_error = api.Context.raise_on_device_error


@pytest.fixture
def fake(monkeypatch):
    ctx = FakeCtx()
    state = {"adjoint_status": L.RF_OK}
    monkeypatch.setattr(api.Context, "get", classmethod(lambda cls, device=None: ctx))

    def rf_project(raw5, eps, delta, **kw):
        return raw5.clone(), torch.zeros(raw5.shape[1:], dtype=torch.uint8)

    def rf_sweep_forward(proj5, eps, src, h, opts=None, **kw):
        max_sweeps = opts.max_sweeps if opts is not None else 64
        # a 16^2 grid needs more than one directional sweep from a corner source
        ctx.pending = L.RF_ERR_NOT_CONVERGED if max_sweeps < 4 else L.RF_OK
        T = torch.ones(src.shape)
        return T, api.Record(torch.zeros(src.shape, dtype=torch.uint8), torch.ones(src.shape),
                             torch.zeros(proj5.shape))

    def rf_adjoint(src, T, rec, g, **kw):
        ctx.pending = state["adjoint_status"]
        return torch.zeros((5,) + tuple(T.shape)), None

    def rf_project_backward(raw5, clip, eps, delta, gproj, **kw):
        return gproj.clone()

    for name, fn in dict(rf_project=rf_project, rf_sweep_forward=rf_sweep_forward, rf_adjoint=rf_adjoint,
                         rf_project_backward=rf_project_backward).items():
        monkeypatch.setattr(api, name, fn)
    return state


def _inputs():
    raw = torch.zeros((5, 16, 16))
    raw[0] = raw[2] = 1.0
    src = torch.zeros((16, 16), dtype=torch.uint8)
    src[0, 0] = 1
    return raw.requires_grad_(True), src


def test_forward_not_converged_raises(fake):
    raw, src = _inputs()
    with pytest.raises(L.RFError) as e:
        autograd.rf_solve(raw, src, 0.1, opts=api.make_opts(max_sweeps=1))
    assert e.value.status == L.RF_ERR_NOT_CONVERGED
    # the same call with room to converge goes through
    T = autograd.rf_solve(raw, src, 0.1, opts=api.make_opts(max_sweeps=64))
    assert T.shape == (16, 16)


def test_backward_timeout_raises(fake):
    raw, src = _inputs()
    T = autograd.rf_solve(raw, src, 0.1)
    fake["adjoint_status"] = L.RF_ERR_TIMEOUT
    with pytest.raises(L.RFError) as e:
        T.sum().backward()
    assert e.value.status == L.RF_ERR_TIMEOUT


def test_sweep_solve_surfaces_both(fake):
    proj = torch.zeros((5, 16, 16), requires_grad=True)
    src = torch.zeros((16, 16), dtype=torch.uint8)
    with pytest.raises(L.RFError):
        autograd.SweepSolve.apply(proj, src, 0.1, 1e-6, "ordered", api.make_opts(max_sweeps=2))
    T = autograd.SweepSolve.apply(proj, src, 0.1, 1e-6, "ordered", None)
    fake["adjoint_status"] = L.RF_ERR_TIMEOUT
    with pytest.raises(L.RFError):
        T.sum().backward()
