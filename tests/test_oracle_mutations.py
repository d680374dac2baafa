"""Mutation check of the oracle's pins (CPU only).

Each mutation below plants one plausible mistake in a copy of the oracle:
- a dropped term;
- a wrong sign, index or constant;
- a transposed operand.

The test then runs the pin suite (tests/test_oracle_pins.py) against that copy,
which must fail. The reproduction of the stored golden step is left out of that
run: it was written by the oracle itself, so it pins nothing against the paper.
A mutation that survives means a part of the oracle that no pin ties to the
paper or to the mathematics. The mutations run as parallel
subprocesses on copies under a temporary directory; the oracle in the repository
is never touched.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file under oracle/, original text, mutated text); each original text
# occurs exactly once in its file.
MUTATIONS = [
    ("hash primes transposed (Sec. 2.1, spatial hash)", "encoding.py",
     "np.uint32(2654435761), np.uint32(805459861)",
     "np.uint32(805459861), np.uint32(2654435761)"),
    ("dense-level index stride N + 2 instead of N + 1 (Sec. 2.1, multiresolution grid)", "encoding.py",
     "s = np.uint32(n + 1)",
     "s = np.uint32(n + 2)"),
    ("trilinear corner weight swapped (Sec. 2.1)", "encoding.py",
     "(w64[:, k] if b[k] else (1.0 - w64[:, k]))",
     "((1.0 - w64[:, k]) if b[k] else w64[:, k])"),
    ("LayerNorm variance not normalised by the group size (Eq. 2)", "field.py",
     "var = ((hg - mean) ** 2).mean(axis=-1, keepdims=True)",
     "var = ((hg - mean) ** 2).sum(axis=-1, keepdims=True)"),
    ("LayerNorm backward projection term with the wrong sign (Eq. 2)", "field.py",
     "- hh * (dhhat * hh).mean(axis=-1, keepdims=True))",
     "+ hh * (dhhat * hh).mean(axis=-1, keepdims=True))"),
    ("ReLU mask of the MLP backward taken from the wrong layer", "field.py",
     "dz = da * (zs[k - 1] > 0.0)",
     "dz = da * (zs[k] > 0.0)"),
    ("detector pixel centre offset dropped (Sec. 2.2)", "geometry.py",
     "ou = ((i + f32(0.5)) - half_nu) * f32(du)",
     "ou = (i - half_nu) * f32(du)"),
    ("detector centre cosine and sine transposed (Sec. 2.2)", "geometry.py",
     "0.5 - ddet * ct, 0.5 - ddet * st, 0.5,",
     "0.5 - ddet * st, 0.5 - ddet * ct, 0.5,"),
    ("SplitMix64 second shift off by one", "geometry.py",
     "(z ^ (z >> np.uint64(27)))",
     "(z ^ (z >> np.uint64(28)))"),
    ("Beer-Lambert sum averaged instead of summed (Eq. 1)", "train.py",
     "* delta[hit].astype(np.float64)[:, None]).sum(axis=1)",
     "* delta[hit].astype(np.float64)[:, None]).mean(axis=1)"),
    ("Adam first-moment bias correction dropped", "train.py",
     "mhat = m / (1.0 - cfg.beta1 ** t)",
     "mhat = m"),
    ("projector voxel-centre offset dropped (Sec. 3.1)", "project.py",
     "pc = x * f32(D) - f32(0.5)",
     "pc = x * f32(D)"),
    ("FFT mask statistic taken on the low band (Sec. 2.3)", "mask.py",
     "hi = P[high].sum(axis=0)",
     "hi = P[~high].sum(axis=0)"),
    ("SSIM contrast constant built from K1 (Wang et al. 2004)", "ssim.py",
     "c2 = (K2 * data_range) ** 2",
     "c2 = (K1 * data_range) ** 2"),
    ("SSIM Gaussian window without the factor 2 in its exponent", "ssim.py",
     "g = np.exp(-(t * t) / (2.0 * sigma * sigma))",
     "g = np.exp(-(t * t) / (sigma * sigma))"),
    ("SSIM covariance factor 2 dropped", "ssim.py",
     "((2.0 * mx * my + c1) * (2.0 * cxy + c2))",
     "((2.0 * mx * my + c1) * (cxy + c2))"),
    ("SSIM window not normalised to sum 1", "ssim.py",
     "return g / g.sum()",
     "return g / g.max()"),
    ("L1 loss gradient with the wrong sign (Eq. 3)", "train.py",
     "return float(np.mean(np.abs(r))), np.sign(r) / R",
     "return float(np.mean(np.abs(r))), -np.sign(r) / R"),
    ("Adam second-moment bias correction dropped", "train.py",
     "vhat = v / (1.0 - cfg.beta2 ** t)",
     "vhat = v"),
    ("Adam epsilon moved inside the square root", "train.py",
     "(np.sqrt(vhat) + cfg.adam_eps)",
     "np.sqrt(vhat + cfg.adam_eps)"),
    ("sigmoid derivative missing its (1 - mu) factor", "field.py",
     "dz = (dmu * mu * (1.0 - mu))[:, None]",
     "dz = (dmu * mu)[:, None]"),
    ("channel mask not applied after the LN affine step (Sec. 2.3)", "field.py",
     "y = (gamma * hhat + beta) * mask",
     "y = (gamma * hhat + beta)"),
    ("LN gamma gradient without the normalized features", "field.py",
     "dgamma = np.sum(g * hhat, axis=0)",
     "dgamma = np.sum(g, axis=0)"),
    ("slab clip taking the nearest entry instead of the farthest", "geometry.py",
     "near = np.where(nz, np.maximum(near, t0), near)",
     "near = np.where(nz, np.minimum(near, t0), near)"),
    ("sample positions at stratum starts instead of midpoints", "geometry.py",
     "ti = (np.arange(N, dtype=np.float32) + f32(0.5))[None, :]",
     "ti = np.arange(N, dtype=np.float32)[None, :]"),
    ("hash scatter without the trilinear weights", "encoding.py",
     "contrib = (w[:, l, :] * dh[:, l * F + f][:, None]).ravel()",
     "contrib = np.broadcast_to(dh[:, l * F + f][:, None], w[:, l, :].shape).ravel()"),
    ("projector trilinear weights swapped", "project.py",
     "w = np.prod(np.where(b[None, :] == 1, fr, 1.0 - fr), axis=1)",
     "w = np.prod(np.where(b[None, :] == 1, 1.0 - fr, fr), axis=1)"),
    ("FFT mask statistic without removing each channel's mean", "mask.py",
     "h = h - h.mean(axis=(0, 1, 2), keepdims=True)",
     "h = h"),
    ("one LN group and per-level groups swapped (Sec. 2.3)", "field.py",
     "return 1 if cfg.norm == 1 else (cfg.n_levels if cfg.norm == 2 else 0), D",
     "return cfg.n_levels if cfg.norm == 1 else (1 if cfg.norm == 2 else 0), D"),
    ("voxel-loss gradient with the wrong sign (Eq. 2)", "train.py",
     "grad = flatten(field_backward(p, cache, np.sign(r) / P, cfg))",
     "grad = flatten(field_backward(p, cache, -np.sign(r) / P, cfg))"),
    ("voxel read-out at cell corners instead of centres", "geometry.py",
     "g = (np.arange(D, dtype=np.float32) + f32(0.5)) / f32(D)",
     "g = np.arange(D, dtype=np.float32) / f32(D)"),
    ("view angles spread over n_views - 1 intervals", "geometry.py",
     "theta = angle0_rad + (v * span_rad) / n_views",
     "theta = angle0_rad + (v * span_rad) / (n_views - 1)"),
    ("level resolutions without the guard against exp() landing below N_max", "encoding.py",
     "return [int(math.floor(base_res * math.exp(l * step) + 1e-9)) for l in range(L)]",
     "return [int(math.floor(base_res * math.exp(l * step))) for l in range(L)]"),
    # The measurement model lives with the seeded input generators, which feed both
    # sides; a path with a "/" is taken relative to the repository root.
    ("Poisson rate I0 e^+A instead of I0 e^-A", "synthetic/__init__.py",
     "I = rng.poisson(I0 * np.exp(-np.asarray(A_clean, dtype=np.float64)))",
     "I = rng.poisson(I0 * np.exp(np.asarray(A_clean, dtype=np.float64)))"),
    ("count floor max(I, 1) dropped", "synthetic/__init__.py",
     "return (-np.log(np.maximum(I, 1) / I0)).astype(np.float32)",
     "return (-np.log(I / I0)).astype(np.float32)"),
    ("measured line integral not normalised by I0", "synthetic/__init__.py",
     "return (-np.log(np.maximum(I, 1) / I0)).astype(np.float32)",
     "return (-np.log(np.maximum(I, 1))).astype(np.float32)"),
]

_IGNORE = shutil.ignore_patterns("__pycache__", "*.pyc")
_SELF_PIN = "tests/test_oracle_pins.py::test_oracle_reproduces_its_stored_step"


def _mutated_tree(base, idx, fname, old, new):
    root = os.path.join(base, f"m{idx:02d}")
    for d in ("oracle", "synthetic", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(root, d), ignore=_IGNORE)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), root)
    path = os.path.join(root, fname) if "/" in fname else os.path.join(root, "oracle", fname)
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not unique in {path}: {old!r}"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    return root


def _pins_fail(root):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-m", "not gpu", "-p", "no:cacheprovider", "--deselect", _SELF_PIN],
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    # exit 1: a pin failed; anything else (collection or usage error) is not a caught mutation
    return r.returncode == 1, r.stdout[-400:]


def test_every_mutation_fails_a_pin(tmp_path):
    roots = [_mutated_tree(str(tmp_path), i, f, o, n) for i, (_, f, o, n) in enumerate(MUTATIONS)]
    workers = max(1, min(len(roots), (os.cpu_count() or 2) // 2))
    with ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(_pins_fail, roots))
    survivors = [(m[0], tail) for m, (caught, tail) in zip(MUTATIONS, results) if not caught]
    assert not survivors, "mutations not caught by any pin:\n" + "\n".join(
        f"- {name}\n{tail}" for name, tail in survivors)


def test_unmutated_copy_passes(tmp_path):
    """The copied tree itself passes the pins, so a failure above comes from the mutation."""
    root = _mutated_tree(str(tmp_path), 0, "train.py", "mhat = m / (1.0 - cfg.beta1 ** t)",
                         "mhat = m / (1.0 - cfg.beta1 ** t)")
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x",
                        "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:]
