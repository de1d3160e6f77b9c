"""The indicator oracle pinned on the CPU: hand-written backpropagation
against central finite differences in FP64, the BF16 rounding against its
definition, and the feature and label definitions on cases with known
answers."""
import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W


def test_backprop_matches_central_differences(oracle_mod):
    from oracle import gate
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, gate.NPARAM)
    X = rng.uniform(-1, 1, (17, gate.NIN))
    y = (rng.uniform(size=17) > 0.5).astype(float)
    L, g = gate.loss_and_grad(theta, X, y, w1=3.0, w0=0.7)
    idx = rng.choice(gate.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [gate.NPARAM - 1, 0]])  # include b3 and W1[0,0]
    for i in idx:
        e = np.zeros(gate.NPARAM)
        e[i] = 1e-6
        Lp, _ = gate.loss_and_grad(theta + e, X, y, 3.0, 0.7)
        Lm, _ = gate.loss_and_grad(theta - e, X, y, 3.0, 0.7)
        fd = (Lp - Lm) / 2e-6
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_bf16_rounding_definition(oracle_mod):
    from oracle import gate
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.1415926, 0.0])
    r = gate.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0  # exactly halfway: ties to even mantissa -> 1.0
    assert r[1] == 1.0
    assert r[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert r[3] == -2.5 and r[5] == 0.0
    assert abs(r[4] - 3.1415926) <= 2 ** -8 * 4


def test_features_of_uniform_and_step_states(oracle_mod):
    from oracle import gate
    U = W.random_subgrids(1, 3)[0]
    U[:] = U[:, :1, :1, :1]  # uniform sub-grid
    X = gate.features(U[None], 5 / 3)
    assert X.shape == (512, 54) and np.all(X == 0.0)
    # density doubles for x >= 7 (interior index 4): a cell just left of the
    # jump sees +1/3 at its three +x neighbours of the density block
    Ug, h, lo = W.sedov_box(8)
    Ug[0, :, :, 4:] *= 2.0
    Up = np.pad(Ug, ((0, 0), (3, 3), (3, 3), (3, 3)), mode="wrap")
    X = gate.features(Up[None], 5 / 3).reshape(8, 8, 8, 54)
    row = X[0, 0, 3, :27].reshape(3, 3, 3)  # cell x = 3 (interior), density part, [dz][dy][dx]
    assert np.allclose(row[:, :, 2], 1.0 / 3.0) and np.allclose(row[:, :, :2], 0.0)


def test_labels_flag_extrema_not_uniform_or_linear(oracle_mod):
    from oracle import gate
    U = W.random_subgrids(1, 3)[0]
    U[:] = U[:, :1, :1, :1]
    assert gate.labels(U[None], 5 / 3).sum() == 0  # uniform: limiter changes nothing
    U[0, 6, 6, 6] *= 1.5  # a density spike: limiter active around it
    lab = gate.labels(U[None], 5 / 3).reshape(8, 8, 8)
    assert lab[3, 3, 3] == 1 and lab[0, 7, 0] == 0


def test_inference_rounds_inputs_and_first_hidden_layer(oracle_mod):
    """forward_infer rounds x and h1 to BF16 and nothing else: with W1 the
    identity on the first two features, one hidden unit passing through to
    the output, the output is exactly sigmoid of the twice-rounded input."""
    from oracle import gate
    p = {name: np.zeros(shape) for name, shape in gate.SIZES}
    p["W1"][0, 0] = 1.0
    p["W1"][1, 1] = 0.5
    p["W2"][0, 0] = 1.0
    p["W2"][0, 1] = 0.25
    p["w3"][0] = 1.0
    theta = np.concatenate([p[name].ravel() for name, _ in gate.SIZES])
    x = np.zeros((3, gate.NIN))
    x[0, 0] = 1.0 + 2.0 ** -9          # halfway between two BF16 values: ties to even -> 1
    x[1, 0] = 1.0 + 3 * 2.0 ** -9      # above halfway -> 1 + 2^-7
    x[2, 0], x[2, 1] = 0.3, 0.7
    out = gate.forward_infer(theta, x)

    def b(v):
        return float(gate.bf16_round(np.array([v]))[0])

    want = [b(x[i, 0]) + 0.25 * b(0.5 * b(x[i, 1])) for i in range(3)]
    assert b(x[0, 0]) == 1.0 and b(x[1, 0]) == 1.0 + 2.0 ** -7
    assert np.array_equal(np.log(out / (1 - out)).round(12), np.array(want).round(12))
    # exact activations differ where the rounding matters
    ref, _ = gate.forward(theta, x)
    assert not np.allclose(out, ref, rtol=0, atol=1e-9)
