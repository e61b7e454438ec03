"""Plant plausible mistakes in copies of the U-Net oracle (on the CPU) and check that the
pins of test_unet_oracle_pins.py catch every one: a flipped kernel, a dropped bias or ReLU
mask, a wrong concatenation slice, a transposed tap, a wrong pooling rule, a wrong Adam
correction, a wrong BF16 tie rule.  Each mutant is a patched copy of unet_oracle.py run
against the pins in a subprocess."""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "unet_oracle.py")
PINS = os.path.join(ROOT, "tests", "test_unet_oracle_pins.py")

# (name, original text, mutated text); each original must occur in the source
MUTANTS = [
    ("convolution_instead_of_correlation",
     "y += xp[:, dh:dh + H, dw:dw + W, :] @ w[:, dh, dw, :].T",
     "y += xp[:, dh:dh + H, dw:dw + W, :] @ w[:, 2 - dh, 2 - dw, :].T"),
    ("bias_dropped", "y = np.broadcast_to(b, (n, H, W, w.shape[0])).copy()",
     "y = np.zeros((n, H, W, w.shape[0]))"),
    ("relu_mask_dropped_in_backward", "            dz = dh * (out > 0)\n            dx, gw, _ = conv3x3_backward(A[f\"{name}_in\"], P[name][0], q(dz))\n            G[name] = (gw, dz.sum(axis=(0, 1, 2)))\n            dh = dx\n        c_up",
     "            dz = dh\n            dx, gw, _ = conv3x3_backward(A[f\"{name}_in\"], P[name][0], q(dz))\n            G[name] = (gw, dz.sum(axis=(0, 1, 2)))\n            dh = dx\n        c_up"),
    ("skip_slice_swapped", "dskip[l] = dh[..., c_up:]", "dskip[l] = dh[..., :dh.shape[3] - c_up]"),
    ("input_gradient_tap_transposed", "dxp[:, dh:dh + H, dwi:dwi + W, :] += dy @ w[:, dh, dwi, :]",
     "dxp[:, dh:dh + H, dwi:dwi + W, :] += dy @ w[:, dwi, dh, :]"),
    ("pool_gradient_to_every_maximum", "hit = (v == y) & ~taken", "hit = (v == y)"),
    ("upsample_gradient_not_summed", "return dy.reshape(n, H2 // 2, 2, W2 // 2, 2, c).sum(axis=(2, 4))",
     "return dy[:, ::2, ::2, :]"),
    ("adam_bias_correction_dropped", "mh = m / (1 - b1 ** step)", "mh = m"),
    ("loss_scale", "inv = 1.0 / (n * H * W * c)", "inv = 1.0 / (n * H * W)"),
    ("bf16_ties_away_from_zero", "u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16",
     "u = ((u + 0x8000) >> 16) << 16"),
]


def test_every_mutant_text_is_present():
    src = open(SRC).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) >= 1, name


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new):
    src = open(SRC).read()
    with tempfile.TemporaryDirectory() as d:
        os.makedirs(os.path.join(d, "oracle"))
        os.makedirs(os.path.join(d, "tests"))
        open(os.path.join(d, "oracle", "__init__.py"), "w").close()
        with open(os.path.join(d, "oracle", "unet_oracle.py"), "w") as f:
            f.write(src.replace(old, new))
        shutil.copy(PINS, os.path.join(d, "tests", "test_unet_oracle_pins.py"))
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                            "tests/test_unet_oracle_pins.py"], cwd=d, capture_output=True,
                           text=True, timeout=600)
    assert r.returncode == 1, f"{name}: the pins did not fail\n{r.stdout[-2000:]}"
