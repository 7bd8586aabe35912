"""The corrector's CUDA kernels against the FP64 oracle (forward pass, loss,
every parameter gradient, the Adam step, the coarsened index), and training
on pairs generated by the propagation: the loss falls and, on held-out
seeds, coarse steps with the corrector are closer to fine-step BPM than
coarse steps without it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import corrector as oc  # noqa: E402
from paper_1706_02261_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1706_02261_b300 import bpm
    return bpm


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("c_in", [2, 3])
def test_forward_loss_and_gradients_match_oracle(B, c_in):
    dev = torch.device("cuda")
    rng = np.random.default_rng(10 + c_in)
    theta = inputs.corrector_init(c_in, 5) + 0.05 * rng.standard_normal(inputs.corrector_param_count(c_in))
    bsz, h, w = 2, 32, 48
    X = rng.standard_normal((bsz, c_in, h, w)).astype(np.float32)
    T = rng.standard_normal((bsz, 2, h, w)).astype(np.float32)
    corr = B.Corrector(c_in, 4, 64, 64)
    sigma = 0.37
    try:
        corr.set_residual_scale(sigma)
        corr.set_params(theta.astype(np.float32))
        work = corr.get_params(which=1).astype(np.float64)        # BF16-rounded weights used by the kernels
        assert np.max(np.abs(work - theta)) <= 0.01 * np.max(np.abs(theta))
        xd, td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
        out = torch.empty((bsz, 2, h, w), dtype=torch.float32, device=dev)
        corr.forward(xd, out)
        ref_out, _, _ = oc.forward(work, X.astype(np.float64), sigma)
        assert rel(out.cpu().numpy(), ref_out) <= 1e-5
        loss = corr.loss_grad(xd, td)
        g = corr.get_params(which=2).astype(np.float64)
        ref_loss, ref_g = oc.loss_and_grad(work, X.astype(np.float64), T.astype(np.float64), sigma)
        assert loss == pytest.approx(ref_loss, rel=1e-5)
        k = 0
        for o, i in oc.layer_shapes(c_in):       # every layer's weights and biases
            for size in (o * i * 9, o):
                assert rel(g[k:k + size], ref_g[k:k + size]) <= 1e-4
                k += size
    finally:
        corr.free()


def test_adam_step_matches_oracle(B):
    dev = torch.device("cuda")
    rng = np.random.default_rng(3)
    theta = inputs.corrector_init(2, 1) + 0.05 * rng.standard_normal(inputs.corrector_param_count(2))
    X = torch.from_numpy(rng.standard_normal((2, 2, 16, 16)).astype(np.float32)).to(dev)
    T = torch.from_numpy(rng.standard_normal((2, 2, 16, 16)).astype(np.float32)).to(dev)
    corr = B.Corrector(2, 2, 16, 16)
    try:
        corr.set_params(theta.astype(np.float32))
        m = np.zeros(theta.size)
        v = np.zeros(theta.size)
        th = corr.get_params(0).astype(np.float64)
        for t in (1, 2):
            corr.loss_grad(X, T)
            g = corr.get_params(2).astype(np.float64)
            corr.adam(1e-3)
            th, m, v = oc.adam_step(th, g, m, v, t, 1e-3)
            got = corr.get_params(0).astype(np.float64)
            assert np.max(np.abs(got - th)) <= 1e-6 * max(1.0, np.max(np.abs(th)))
    finally:
        corr.free()


def test_coarsen_index(B):
    dev = torch.device("cuda")
    rng = np.random.default_rng(4)
    dn = rng.uniform(0, 0.05, size=(10, 32, 48)).astype(np.float16)
    out = torch.empty((2, 32, 48), dtype=torch.float16, device=dev)
    B.bpm_coarsen_index(torch.from_numpy(dn).to(dev), 4, out)
    torch.cuda.synchronize()
    ref = dn[:8].astype(np.float64).reshape(2, 4, 32, 48).mean(axis=1)
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 2 ** -11 * 0.05      # within FP16 rounding at |dn| <= 0.05


@pytest.mark.parametrize("c_in,min_gain", [(2, 1.05), (3, 1.5)])
def test_training_gains_over_coarse_steps_on_held_out_seeds(B, c_in, min_gain):
    """Train on pairs from seeds 4000-4047 (128^2 x 64 fine slices, 16 coarse
    steps each); on held-out seeds 5000-5005 the field after the volume, coarse
    steps with the corrector versus without, both against fine-step BPM.  The
    2-channel network is the specified one; the 3-channel one also sees the
    averaged index step."""
    from paper_1706_02261_b300 import corrector as C
    dev = torch.device("cuda")
    s = C.Setup(n=128, nz=64, c_in=c_in)
    corr = B.Corrector(s.c_in, 16, s.n, s.n)
    try:
        corr.set_params(inputs.corrector_init(s.c_in, 0).astype(np.float32))
        X, T = C.make_pairs(s, range(4000, 4048), corr, dev)
        sigma = C.residual_scale(corr, X, T)
        corr.set_residual_scale(sigma)
        losses = C.train(corr, X, T, steps=3000, batch=16, lr=1e-3, seed=1, log_every=500)
        if c_in == 3:
            assert losses[-1][1] < 0.5 * losses[0][1], losses
        ev = C.evaluate(s, range(5000, 5006), corr, dev)
        gain = np.mean([r["coarse"] for r in ev]) / np.mean([r["corrected"] for r in ev])
        print(f"c_in={c_in} sigma={sigma:.3e} losses={losses} held-out={ev} gain={gain:.2f}")
        assert gain > min_gain, ev
    finally:
        corr.free()


@pytest.mark.parametrize("c_in,min_gain", [(2, 1.05), (3, 1.5)])
def test_crop_pairs_gain_on_held_out_volumes(B, c_in, min_gain):
    """The workload's recipe at 256^3: pairs as 128^2 crops of full fine-step
    fields (seeds 4000-4011, 256 crops each), held-out volumes 5000-5003
    through coarse steps with and without the corrector, errors against
    fine-step BPM: the field error falls by min_gain, and (3 channels) the
    intensity error falls as well."""
    from paper_1706_02261_b300 import corrector as C
    dev = torch.device("cuda")
    cs = C.CropSetup(n=256, nz=256, crop=128, c_in=c_in)
    corr = B.Corrector(c_in, 32, cs.n, cs.n)
    try:
        corr.set_params(inputs.corrector_init(c_in, 0).astype(np.float32))
        X, T = C.make_crop_pairs(cs, range(4000, 4012), corr, dev, 256, rng_seed=c_in)
        corr.set_residual_scale(C.residual_scale(corr, X, T, batch=32))
        C.train(corr, X, T, steps=3000, batch=32, lr=1e-3, seed=1)
        del X, T
        rows = [C.evaluate_volume(cs, sd, corr, dev) for sd in range(5000, 5004)]
        gain = np.mean([r["coarse_field"] for r in rows]) / np.mean([r["corrected_field"] for r in rows])
        igain = np.mean([r["coarse_intensity"] for r in rows]) / np.mean([r["corrected_intensity"] for r in rows])
        print(f"c_in={c_in} field gain {gain:.2f} intensity gain {igain:.2f} rows={rows}")
        assert gain > min_gain, rows
        if c_in == 3:
            assert igain > 1.2, rows
    finally:
        corr.free()


@pytest.mark.parametrize("c_in,bsz,h,w", [(2, 2, 32, 128), (3, 3, 16, 256)])
def test_tensor_core_gradients_match_fp32_pipes(B, c_in, bsz, h, w):
    """Loss and every parameter gradient from the tensor-core training path
    (BF16 activations and data gradients, FP32 accumulation) against the FP32
    path, which the oracle pins to 1e-4: agreement to the BF16 rounding of
    the operands."""
    dev = torch.device("cuda")
    rng = np.random.default_rng(40 + c_in)
    theta = inputs.corrector_init(c_in, 5) + 0.05 * rng.standard_normal(inputs.corrector_param_count(c_in))
    X = torch.from_numpy(rng.standard_normal((bsz, c_in, h, w)).astype(np.float32)).to(dev)
    T = torch.from_numpy(rng.standard_normal((bsz, 2, h, w)).astype(np.float32)).to(dev)
    corr = B.Corrector(c_in, 4, h, w)
    try:
        corr.set_residual_scale(0.37)
        corr.set_params(theta.astype(np.float32))
        loss32 = corr.loss_grad(X, T)
        g32 = corr.get_params(which=2).astype(np.float64)
        corr.set_train_tensor_cores(True)
        loss_tc = corr.loss_grad(X, T)
        corr.check()
        gtc = corr.get_params(which=2).astype(np.float64)
        print(f"c_in={c_in}: loss {loss32:.6e} / {loss_tc:.6e}")
        assert loss_tc == pytest.approx(loss32, rel=2e-2)
        k = 0
        for o, i in oc.layer_shapes(c_in):
            for size in (o * i * 9, o):
                e = rel(gtc[k:k + size], g32[k:k + size])
                print(f"  block {k}: rel {e:.2e}")
                assert e <= 3e-2, (k, e)
                k += size
    finally:
        corr.free()


def test_tensor_core_training_gains_on_held_out_volumes(B):
    """The crop recipe of the 512^3 workload at 256^3, trained on the tensor
    cores (3 channels): the held-out field error falls as with the FP32
    training path."""
    from paper_1706_02261_b300 import corrector as C
    dev = torch.device("cuda")
    cs = C.CropSetup(n=256, nz=256, crop=128, c_in=3)
    corr = B.Corrector(3, 32, cs.n, cs.n)
    try:
        corr.set_params(inputs.corrector_init(3, 0).astype(np.float32))
        X, T = C.make_crop_pairs(cs, range(4000, 4012), corr, dev, 256, rng_seed=3)
        corr.set_residual_scale(C.residual_scale(corr, X, T, batch=32))
        corr.set_train_tensor_cores(True)
        C.train(corr, X, T, steps=3000, batch=32, lr=1e-3, seed=1)
        corr.check()
        del X, T
        rows = [C.evaluate_volume(cs, sd, corr, dev) for sd in range(5000, 5004)]
        gain = np.mean([r["coarse_field"] for r in rows]) / np.mean([r["corrected_field"] for r in rows])
        print(f"tensor-core training: field gain {gain:.2f} rows={rows}")
        assert gain > 1.5, rows
    finally:
        corr.free()


@pytest.mark.parametrize("c_in,h,w", [(2, 32, 128), (3, 16, 256)])
def test_tensor_core_forward_matches_bf16_activation_oracle(B, c_in, h, w):
    """The tcgen05 inference engine (BF16 activations and weights, FP32
    accumulation in tensor memory) against the oracle with the same BF16
    rounding of every convolution input; tiles of 128 pixels, circular
    halos across the row ends and the image edges."""
    dev = torch.device("cuda")
    rng = np.random.default_rng(20 + c_in)
    theta = inputs.corrector_init(c_in, 5) + 0.05 * rng.standard_normal(inputs.corrector_param_count(c_in))
    bsz = 2
    X = rng.standard_normal((bsz, c_in, h, w)).astype(np.float32)
    corr = B.Corrector(c_in, 4, 32, 256)
    sigma = 0.37
    try:
        corr.set_residual_scale(sigma)
        corr.set_params(theta.astype(np.float32))
        work = corr.get_params(which=1).astype(np.float64)
        xd = torch.from_numpy(X).to(dev)
        out = torch.empty((bsz, 2, h, w), dtype=torch.float32, device=dev)
        corr.set_tensor_cores(True)
        corr.forward(xd, out)
        corr.check()
        f_gpu = (out.cpu().numpy().astype(np.float64) - X[:, :2]) / sigma
        ref, _, _ = oc.forward(work, X.astype(np.float64), sigma, act_bf16=True)
        f_ref = (ref - X[:, :2]) / sigma
        e = rel(f_gpu, f_ref)
        corr.set_tensor_cores(False)
        corr.forward(xd, out)
        f_fp32 = (out.cpu().numpy().astype(np.float64) - X[:, :2]) / sigma
        print(f"c_in={c_in} {h}x{w}: tensor cores vs BF16-activation oracle {e:.2e}; "
              f"FP32 pipes vs the same {rel(f_fp32, f_ref):.2e}")
        assert e <= 5e-4
    finally:
        corr.free()


def test_apply_on_tensor_cores_agrees_with_fp32_pipes_at_512(B):
    from paper_1706_02261_b300 import corrector as C
    dev = torch.device("cuda")
    s = C.Setup(n=512, nz=8, c_in=3)
    corr = B.Corrector(3, 1, 512, 512)
    try:
        rng = np.random.default_rng(2)
        corr.set_params((inputs.corrector_init(3, 0) + 0.02 * rng.standard_normal(inputs.corrector_param_count(3)))
                        .astype(np.float32))
        corr.set_residual_scale(0.05)
        dnc = torch.from_numpy(rng.uniform(0, 0.05, (512, 512)).astype(np.float16)).to(dev)
        e0 = torch.from_numpy(np.exp(1j * rng.uniform(0, 6, (512, 512))).astype(np.complex64)).to(dev)
        ea, eb = e0.clone(), e0.clone()
        corr.set_tensor_cores(True)
        corr.apply(ea, dnc, s.dn_scale)
        corr.check()
        corr.set_tensor_cores(False)
        corr.apply(eb, dnc, s.dn_scale)
        torch.cuda.synchronize()
        d = float(torch.linalg.vector_norm(ea - eb) / torch.linalg.vector_norm(eb - e0))
        print(f"512^2 apply: tensor cores vs FP32 pipes, relative to the correction: {d:.2e}")
        assert d <= 2e-2
    finally:
        corr.free()
