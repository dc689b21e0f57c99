"""The training-loop integration (paper_2206_15397_gb300.optim.RandomizedKFAC):
hooks feed the layers' inputs and output gradients to the library's EA
update, the factors are inverted on the T_KI schedule and every step's
gradients come back preconditioned. Checked against the FP64 oracle built from
the same captured tensors (torch's forward/backward, not the library) and the
same Gaussian test matrices (the library draws them on the device from the
optimizer's per-factor seeds; the host generator evaluates the same definition)."""
import numpy as np
import pytest

import oracle
from paper_2206_15397_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def optim():
    from paper_2206_15397_gb300 import build
    build.build()
    from paper_2206_15397_gb300 import optim as o
    return o


def model_and_data(seed=0):
    torch.manual_seed(seed)
    model = torch.nn.Sequential(torch.nn.Linear(40, 64), torch.nn.Tanh(), torch.nn.Linear(64, 10, bias=False)).cuda()
    x = torch.randn(128, 40, device="cuda")
    y = torch.randn(128, 10, device="cuda")
    return model, x, y


@pytest.mark.parametrize("method", ["srevd", "rsvd"])
def test_one_step_matches_oracle(optim, method):
    model, x, y = model_and_data()
    r, p, q, lam, rho = 16, 6, 1, 0.1, 0.9
    pre = optim.RandomizedKFAC(model, rank=r, oversample=p, power_iters=q, damping=lam, rho=rho, t_update=1,
                               t_invert=1, method=method, seed=5)
    acts, gouts = [], []
    lins = [m for m in model.modules() if isinstance(m, torch.nn.Linear)]
    hs = [m.register_forward_pre_hook(lambda mod, a: acts.append(a[0].detach().double().cpu().numpy())) for m in lins]
    hs += [m.register_full_backward_hook(lambda mod, gi, go: gouts.append(go[0].detach().double().cpu().numpy()))
           for m in lins]
    loss = torch.nn.functional.mse_loss(model(x), y)
    loss.backward()
    gouts = gouts[::-1]  # backward visits the layers last to first
    grads = [torch.cat([m.weight.grad, m.bias.grad[:, None]], 1) if m.bias is not None else m.weight.grad
             for m in lins]
    grads = [g.double().cpu().numpy() for g in grads]
    pre.step()
    for h in hs:
        h.remove()
    assert pre.status()[0] == 0
    invert = oracle.invert if method == "srevd" else oracle.invert_rsvd
    n = x.shape[0]
    for li, (m, a, g, j) in enumerate(zip(lins, acts, gouts, grads)):
        abar = np.hstack([a, np.ones((n, 1))]) if m.bias is not None else a
        fa = oracle.ea_update(np.zeros((abar.shape[1],) * 2), abar.T, rho)
        fg = oracle.ea_update(np.zeros((g.shape[1],) * 2), (n * g).T, rho)
        inv = []
        for side, f in enumerate((fa, fg)):
            d = f.shape[0]
            k = min(r, d) + p
            om = (inputs.seeded_omega(optim.omega_seed(5, 0, 2 * li + side), d, k).astype(np.float64) if k < d
                  else np.zeros((d, k)))
            inv.append(invert(f.astype(np.float32).astype(np.float64), om, min(r, d), q, lam))
        (ua, _, ca), (ug, _, cg) = inv
        want = oracle.precondition(j, ua, ca, ug, cg, lam)
        got = torch.cat([m.weight.grad, m.bias.grad[:, None]], 1) if m.bias is not None else m.weight.grad
        got = got.double().cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want), np.linalg.norm(got - want) / np.linalg.norm(want)


def test_training_with_the_amortised_schedule_reduces_the_loss(optim):
    model, x, y = model_and_data(1)
    pre = optim.RandomizedKFAC(model, rank=16, oversample=6, damping=0.1, t_update=2, t_invert=5)
    sgd = torch.optim.SGD(model.parameters(), lr=0.05)
    losses = []
    for _ in range(30):
        sgd.zero_grad()
        loss = torch.nn.functional.mse_loss(model(x), y)
        loss.backward()
        pre.step()
        sgd.step()
        losses.append(float(loss.detach()))
    assert pre.status()[0] == 0
    assert losses[-1] < 0.7 * losses[0], losses
