"""Host logic of the FWI driver on the CPU, with a stand-in for the FDTD context: a
quadratic misfit J(m) = 1/2 sum w (m - m_true)^2 in the variables (eps_r, sigma / sigma_ref),
whose gradient is known exactly.  Checks the L-BFGS iteration's bookkeeping: an L-BFGS step
whose first trial passes Armijo costs exactly one misfit-and-gradient evaluation (its gradient
is reused as the next iteration's), the evaluation counts in the history match the calls made,
and the iteration converges."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2506_20513_gb300 import fwi as F  # noqa: E402
from paper_2506_20513_gb300.workloads import GridSpec  # noqa: E402


class QuadraticFD:
    """The parts of FDTD that the driver uses, with a quadratic misfit."""

    def __init__(self, ny=12, nx=16, seed=3):
        rng = np.random.default_rng(seed)
        self.device = torch.device("cpu")
        self.shape = (ny, nx)
        self.grid = GridSpec(nx=nx, ny=ny, npml=2, nt=50, dx=0.01, dy=0.01, dt=1e-11)
        self.eps_true = torch.tensor(4.0 + rng.random((ny, nx)), dtype=torch.float32)
        self.sig_true = torch.tensor(0.005 + 0.01 * rng.random((ny, nx)), dtype=torch.float32)
        self.w_eps = torch.tensor(1.0 + rng.random((ny, nx)), dtype=torch.float64)
        self.w_sig = torch.tensor(1.0 + rng.random((ny, nx)), dtype=torch.float64)
        self.calls = {"misfit": 0, "gradient": 0}

    def _terms(self, eps, sig):
        de = eps.double() - self.eps_true.double()
        ds = (sig.double() - self.sig_true.double()) / 1e-2
        return de, ds

    def misfit(self, eps, sig, wav, obs, out=None):
        self.calls["misfit"] += 1
        de, ds = self._terms(eps, sig)
        J = 0.5 * float((self.w_eps * de * de).sum() + (self.w_sig * ds * ds).sum())
        t = out if out is not None else torch.empty(1, dtype=torch.float64)
        t[0] = J
        return t

    def misfit_and_gradient(self, eps, sig, wav, obs):
        self.calls["gradient"] += 1
        de, ds = self._terms(eps, sig)
        J = 0.5 * float((self.w_eps * de * de).sum() + (self.w_sig * ds * ds).sum())
        ge = (self.w_eps * de).float()
        gs = (self.w_sig * ds / 1e-2).float()  # dJ/dsigma in S/m
        return torch.tensor([J], dtype=torch.float64), ge, gs

    def forward_model(self, eps, sig, wav, illumination=False):
        return None, torch.ones(self.shape)


@pytest.fixture
def no_cuda_sync(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def run(fd, iters, **cfg):
    mask = torch.ones(fd.shape)
    drv = F.FWI(fd, lambda f0: None, mask, F.FWIConfig(bands=((4e8, iters),), **cfg))
    e0 = fd.eps_true + 0.5
    s0 = fd.sig_true * 0.5
    return drv.run(e0, s0)


def test_accepted_lbfgs_steps_cost_one_evaluation(no_cuda_sync):
    fd = QuadraticFD()
    _, _, hist = run(fd, 8)
    total = fd.calls["misfit"] + fd.calls["gradient"]
    # the history accounts for every call except the gradient at the start of the band
    assert sum(hist.evaluations) == total - 1
    # after the first (steepest-descent, backtracking) iteration, a step accepted at its first
    # trial costs exactly one evaluation
    assert hist.evaluations[0] >= 2
    assert hist.evaluations[1:] == [1] * (len(hist.evaluations) - 1)  # alpha = 1 on a quadratic
    # one gradient per iteration at most (reused or computed once at the accepted point)
    assert fd.calls["gradient"] <= 1 + len(hist.evaluations)
    # forward-equivalent passes: a misfit-only evaluation is one time loop, a gradient two
    assert sum(hist.passes) == fd.calls["misfit"] + 2 * fd.calls["gradient"] - 2
    assert hist.passes[1:] == [2] * (len(hist.passes) - 1)


def test_iteration_converges_on_the_quadratic(no_cuda_sync):
    fd = QuadraticFD()
    eps, sig, hist = run(fd, 30)
    assert hist.misfit[-1] < 1e-3 * hist.misfit[0]
    assert float((eps - fd.eps_true).abs().max()) < 0.05


def test_adam_stage_schedule():
    from paper_2506_20513_gb300.adam import AdamConfig, Stage, stage_of
    st = (Stage(3, 0.2, 0.0), Stage(2, 0.1, 1e-4))
    assert [stage_of(st, e) for e in range(6)] == [0, 0, 0, 1, 1, -1]
    # the default is the cross-hole schedule: eps_r alone for 50 epochs, then both
    d = AdamConfig().stages
    assert d[0].epochs == 50 and d[0].lr_sig == 0.0 and d[1].lr_sig > 0.0


class HalfwayPreconditioner:
    """Proposes half of the remaining update at every stage; a stage in ``bad`` proposes a
    step away from the truth instead (its misfit rises, so the driver rejects it)."""

    def __init__(self, fd, bad=()):
        self.fd, self.bad, self.stages = fd, set(bad), []

    def update(self, ge, gs, eps, illum, stage=0):
        self.stages.append(stage)
        f = -1.0 if stage in self.bad else 0.5
        # eps and sigma of the driver's current model from the quadratic's gradients
        de = -ge.double() / self.fd.w_eps
        ds = -gs.double() * 1e-2 / self.fd.w_sig * 1e-2
        return (f * de).float(), (f * ds).float()


def test_learned_stage_counts_kept_updates(no_cuda_sync):
    fd = QuadraticFD()
    pre = HalfwayPreconditioner(fd)
    mask = torch.ones(fd.shape)
    drv = F.FWI(fd, lambda f0: None, mask, F.FWIConfig(bands=((4e8, 4),), learned_max=0),
                preconditioner=pre)
    _, _, hist = drv.run(fd.eps_true + 0.5, fd.sig_true * 0.5)
    # no cap: every learned update lowers the quadratic misfit: all kept, stage = updates kept
    # so far
    assert pre.stages == [0, 1, 2, 3]
    assert hist.learned == [True] * 4


def test_rejected_stage_ends_the_learned_updates(no_cuda_sync):
    fd = QuadraticFD()
    pre = HalfwayPreconditioner(fd, bad={1})
    mask = torch.ones(fd.shape)
    drv = F.FWI(fd, lambda f0: None, mask, F.FWIConfig(bands=((4e8, 5),)), preconditioner=pre)
    _, _, hist = drv.run(fd.eps_true + 0.5, fd.sig_true * 0.5)
    # stage 1 is rejected (every scale tried raises the misfit): L-BFGS for the rest
    assert pre.stages == [0, 1]
    assert hist.learned[:2] == [True, False] and not any(hist.learned[2:])


def test_preconditioner_selects_the_network_of_the_stage():
    from paper_2506_20513_gb300.precond import LearnedPreconditioner

    class Const:
        height, width, device = 4, 6, torch.device("cpu")

        def __init__(self, v):
            self.v = v

        def forward(self, x):
            return torch.full((1, 4, 6, 2), self.v)

    pre = LearnedPreconditioner([Const(1.0), Const(2.0)], npml=2)
    z = torch.zeros(8, 10)
    ill = torch.ones(8, 10)
    got = [float(pre.update(z, z, z + 4.0, ill, stage=k)[0][4, 5]) for k in range(4)]
    # network k after k kept updates; the last network serves every later stage
    assert got == [1.0, 2.0, 2.0, 2.0]
    # a single network serves every stage; the absorbing layer gets no update
    one = LearnedPreconditioner(Const(3.0), npml=2)
    de, ds = one.update(z, z, z + 4.0, ill, stage=5)
    assert float(de[4, 5]) == 3.0 and float(de[0, 0]) == 0.0 and float(ds[1, 1]) == 0.0


def test_learned_max_caps_the_kept_updates(no_cuda_sync):
    fd = QuadraticFD()
    pre = HalfwayPreconditioner(fd)
    mask = torch.ones(fd.shape)
    drv = F.FWI(fd, lambda f0: None, mask, F.FWIConfig(bands=((4e8, 5),), learned_max=2),
                preconditioner=pre)
    _, _, hist = drv.run(fd.eps_true + 0.5, fd.sig_true * 0.5)
    # two updates kept, then the network is not consulted again in the band
    assert pre.stages == [0, 1]
    assert hist.learned == [True, True, False, False, False]


class QuadraticTE(QuadraticFD):
    """The TE calls of a context, over the same quadratic misfit; records the polarisations."""

    def __init__(self):
        super().__init__()
        self.pols = []

    def misfit_te(self, eps, sig, wav, obs, polarisation, out=None):
        self.pols.append(polarisation)
        return self.misfit(eps, sig, wav, obs, out=out)

    def misfit_and_gradient_te(self, eps, sig, wav, obs, polarisation):
        self.pols.append(polarisation)
        return self.misfit_and_gradient(eps, sig, wav, obs)


def test_te_mode_routes_the_driver_to_the_te_calls(no_cuda_sync):
    from paper_2506_20513_gb300.fdtd import TEMode
    fd = QuadraticTE()
    te = TEMode(fd, 1)
    assert te.shape == fd.shape and te.grid is fd.grid   # everything else is the context's
    drv = F.FWI(te, lambda f0: None, torch.ones(fd.shape), F.FWIConfig(bands=((4e8, 20),)))
    eps, _, hist = drv.run(fd.eps_true + 0.5, fd.sig_true * 0.5)
    # every evaluation went through a TE call with the view's polarisation
    assert fd.pols and set(fd.pols) == {1}
    assert len(fd.pols) == fd.calls["misfit"] + fd.calls["gradient"]
    assert hist.misfit[-1] < 1e-3 * hist.misfit[0]
    with pytest.raises(ValueError):
        TEMode(fd, 2)
    with pytest.raises(ValueError):
        te.forward_model(eps, eps, None, illumination=True)
