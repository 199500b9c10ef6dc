"""CUDA FNO (learned warm start) against the FP64 FNO oracle.

The oracle takes the GPU's parameters as the kernels read them (BF16 weights),
so the comparison isolates the kernels' FP32 arithmetic:
  forward                      rel-L2 <= 1e-3
  loss                         rel <= 1e-4
  parameter gradients          cosine >= 0.999 and rel-L2 <= 2e-2 per group
A few Adam steps lower the loss, and a warm start leaves the converged field
unchanged (the solve still stops on the true residual).
"""
import numpy as np
import pytest

from oracle import fno as ofno
from oracle import model, solve
from paper_1708_01663_gb300 import cisor, synth

pytestmark = pytest.mark.gpu
N = 128


def _inputs(B, seed=0):
    fs, us, ts = [], [], []
    ang = synth.plane_wave_angles(B) + 0.3
    u_in = model.plane_waves(ang, N, 1.0 / 8, 2 * np.pi)
    for b in range(B):
        fs.append(synth.ellipse_phantom(N, 4, (0.0, 0.8), seed + b, 0.02))
        us.append(u_in[b])
        ts.append(0.3 * synth.random_field(seed + 50 + b, (N, N)) + 0.5 * fs[-1])
    c = lambda L: np.ascontiguousarray(np.stack(L), dtype=np.complex64)
    return fs, us, ts, c(fs), c(us), c(ts)


def _oracle_params(net):
    flat = np.empty(net.num_params, np.float32)
    net.get_params(flat, as_used=True)
    return cisor.fno_param_dict(flat)


def test_fno_forward_matches_oracle():
    from paper_1708_01663_gb300 import build
    build.build()
    net = cisor.FNO(max_batch=4, seed=7)
    p = _oracle_params(net)
    fs, us, ts, f, u, t = _inputs(2)
    out = np.empty_like(u)
    net.forward(f, u, out)
    for b in range(2):
        ref, _ = ofno.forward(p, fs[b].astype(np.complex64).astype(np.complex128),
                              us[b].astype(np.complex64).astype(np.complex128))
        assert np.linalg.norm(out[b] - ref) / np.linalg.norm(ref) < 1e-3
    net.close()


def test_fno_gradients_match_oracle():
    from paper_1708_01663_gb300 import build
    build.build()
    net = cisor.FNO(max_batch=4, seed=11)
    p = _oracle_params(net)
    fs, us, ts, f, u, t = _inputs(2, seed=3)
    g = np.empty(net.num_params, np.float32)
    loss = net.loss_grad(f, u, t, g)
    c128 = lambda a: a.astype(np.complex64).astype(np.complex128)
    ref_loss, ref_g = ofno.loss_and_grad(p, [c128(x) for x in fs], [c128(x) for x in us], [c128(x) for x in ts])
    assert abs(loss - ref_loss) / ref_loss < 1e-4
    gd = cisor.fno_param_dict(g)
    for k, gr in ref_g.items():
        a = np.concatenate([gd[k].real.ravel(), np.imag(gd[k]).ravel()])
        r = np.concatenate([gr.real.ravel(), np.imag(gr).ravel()])
        nr = np.linalg.norm(r)
        if nr == 0:
            continue
        cos = float(a @ r / (np.linalg.norm(a) * nr))
        assert cos >= 0.999, (k, cos)
        assert np.linalg.norm(a - r) / nr <= 2e-2, (k, np.linalg.norm(a - r) / nr)
    net.close()


def test_fno_training_lowers_loss():
    from paper_1708_01663_gb300 import build
    build.build()
    net = cisor.FNO(max_batch=8, seed=2)
    fs, us, ts, f, u, t = _inputs(8, seed=20)
    t = np.ascontiguousarray((0.5 + 0.2j) * f * u, dtype=np.complex64)   # representable: pointwise in the inputs
    first = net.train_step(f, u, t, 1e-3)
    for _ in range(40):
        last = net.train_step(f, u, t, 1e-3)
    assert last < 0.7 * first
    net.close()


def test_warm_start_keeps_converged_field():
    from paper_1708_01663_gb300 import build
    build.build()
    T = 4
    ang = synth.plane_wave_angles(T)
    rx = synth.circle_receivers(16, 12.0)
    ctx = cisor.Cisor(N, 1.0 / 8, ang, rx, complex_f=True)
    net = cisor.FNO(max_batch=T, seed=4)
    f = synth.ellipse_phantom(N, 4, (0.0, 0.5), 9, 0.02).astype(np.complex64)
    x0 = np.empty((T, N, N), np.complex64)
    net.warm_start(ctx, f, x0)
    assert np.isfinite(x0).all()
    u_cold = np.empty((T, N, N), np.complex64)
    u_warm = np.empty((T, N, N), np.complex64)
    ctx.forward(f, u_out=u_cold, tol=1e-6, max_iter=3000)
    st, info = ctx.forward(f, x0=x0, u_out=u_warm, tol=1e-6, max_iter=3000, x0_mode=1)
    assert info.resid_max <= 1e-6
    prob = model.Problem(N, 1.0 / 8, ang, rx, P=ctx.P)
    ref, _, _ = solve.solve_fields(prob, f.astype(np.complex128), prob.u_in, tol=1e-12)
    assert np.linalg.norm(u_warm - ref) / np.linalg.norm(ref) < 1e-4
    assert np.linalg.norm(u_cold - ref) / np.linalg.norm(ref) < 1e-4
    net.close()
    ctx.close()


def test_trained_warm_start_saves_iterations():
    """A short seeded training run on solver-generated fields (300 phantoms x 32 transmitters of the
    128 x 128 workload, 45 s of Adam) gives a warm start that lowers the mean BiCGSTAB iteration count to
    residual 1e-4 on held-out phantoms, while every solve still stops on the true residual."""
    import torch
    from paper_1708_01663_gb300 import build, train_fno
    build.build()
    dev = torch.device("cuda", 0)
    ang, rx = train_fno.geometry()
    ctx = cisor.Cisor(train_fno.N, train_fno.DELTA, ang, rx)
    fs, usc, u_in = train_fno.generate(ctx, range(300), dev)
    net = cisor.FNO(max_batch=train_fno.T, seed=1714)
    steps, losses = train_fno.train(net, fs, usc, u_in, 0.75)
    del fs, usc
    res = train_fno.evaluate(ctx, net, range(100000, 100016), dev)
    cold, warm = np.mean(res["cold_iters"]), np.mean(res["warm_iters"])
    print(f"steps {steps}, loss {np.mean(losses[:20]):.3f} -> {np.mean(losses[-50:]):.3f}, iterations {cold:.1f} "
          f"-> {warm:.1f}, prediction error {np.mean(res['pred_err']):.3f}")
    assert np.mean(losses[-50:]) < 0.8 * np.mean(losses[:20])
    assert warm < 0.97 * cold
    net.close()
    ctx.close()
