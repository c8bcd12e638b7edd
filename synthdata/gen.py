"""Seeded synthetic inputs shaped like the paper's datasets (Section 4.1).

Each generator returns ``(values, labels)``: ``values`` is a C-contiguous
uint8 array of shape (n, n_values), ``labels`` a uint32 array of shape (n,).
Nothing here encodes, encrypts or otherwise computes the method: the uint8
values play the role of an 8-bit dataset (the paper min-max scales its
Wisconsin features to 8 bits and MNIST/HAM10000 are 8-bit images).

Recipes
-------
uniform  independent uniform bytes and uniform labels (small test rings).
gauss30  real features x ~ N(+1, 1) for class 1 and N(-1, 1) for class 0,
         clipped to [-3, 3] and mapped linearly to 0..255 (Wisconsin shape).
digits   28x28 grey images: each class has a seeded template of 3 strokes and
         one blob; a sample shifts it by up to 2 pixels, scales intensity and
         adds noise (MNIST shape, 10 classes).
lesions  28x28x3 RGB images: a radial colour blob with a class-specific hue,
         radius and ring profile on a skin-coloured background, plus noise,
         flattened as [row][col][channel] (HAM10000 shape, 7 classes).
"""
import numpy as np

from .configs import Config

_GEN_TAGS = {"train": 0, "test": 1}


def _labels(rng, n, priors):
    p = np.asarray(priors, dtype=np.float64)
    p = p / p.sum()
    return rng.choice(len(p), size=n, p=p).astype(np.uint32)


def _gauss30(rng, labels, n_values):
    n = labels.shape[0]
    sign = np.where(labels == 1, 1.0, -1.0)[:, None]
    x = rng.normal(loc=sign, scale=1.0, size=(n, n_values))
    x = np.clip(x, -3.0, 3.0)
    v = np.rint((x + 3.0) * (255.0 / 6.0))
    return v.astype(np.uint8)


def _digit_templates(n_classes, seed):
    trng = np.random.default_rng(seed * 7919 + 17)
    yy, xx = np.mgrid[0:28, 0:28].astype(np.float64)
    out = np.zeros((n_classes, 28, 28))
    for c in range(n_classes):
        img = np.zeros((28, 28))
        for _ in range(3):
            p0 = trng.uniform(5, 23, size=2)
            p1 = trng.uniform(5, 23, size=2)
            d = p1 - p0
            t = ((yy - p0[0]) * d[0] + (xx - p0[1]) * d[1]) / max(d @ d, 1e-9)
            t = np.clip(t, 0.0, 1.0)
            dist = np.hypot(yy - (p0[0] + t * d[0]), xx - (p0[1] + t * d[1]))
            img = np.maximum(img, np.clip(2.2 - dist, 0.0, 1.0))
        bc = trng.uniform(8, 20, size=2)
        br = trng.uniform(2.0, 4.0)
        dist = np.hypot(yy - bc[0], xx - bc[1])
        img = np.maximum(img, np.clip(br - dist, 0.0, 1.0))
        out[c] = img
    return out


def _digits(rng, labels, n_classes, seed):
    tmpl = _digit_templates(n_classes, seed)
    n = labels.shape[0]
    out = np.empty((n, 784), dtype=np.uint8)
    shifts = rng.integers(-2, 3, size=(n, 2))
    gain = rng.uniform(0.75, 1.0, size=n)
    for i in range(n):
        img = np.roll(tmpl[labels[i]], shift=(int(shifts[i, 0]), int(shifts[i, 1])), axis=(0, 1))
        img = img * gain[i] + rng.normal(0.0, 0.08, size=(28, 28))
        out[i] = np.clip(np.rint(img * 255.0), 0, 255).astype(np.uint8).reshape(-1)
    return out


def _lesions(rng, labels, n_classes, seed):
    crng = np.random.default_rng(seed * 104729 + 5)
    hue = crng.uniform(0.0, 1.0, size=(n_classes, 3))
    radius = crng.uniform(5.0, 11.0, size=n_classes)
    ring = crng.uniform(0.0, 1.0, size=n_classes)
    yy, xx = np.mgrid[0:28, 0:28].astype(np.float64)
    skin = np.array([0.85, 0.65, 0.55])
    n = labels.shape[0]
    out = np.empty((n, 2352), dtype=np.uint8)
    centers = rng.uniform(10.0, 18.0, size=(n, 2))
    rscale = rng.uniform(0.8, 1.2, size=n)
    for i in range(n):
        c = labels[i]
        d = np.hypot(yy - centers[i, 0], xx - centers[i, 1]) / (radius[c] * rscale[i])
        body = np.clip(1.0 - d, 0.0, 1.0)
        rim = np.exp(-((d - 0.8) ** 2) / 0.02) * ring[c]
        w = np.clip(body + rim, 0.0, 1.0)[..., None]
        img = skin * (1.0 - w) + hue[c] * w + rng.normal(0.0, 0.05, size=(28, 28, 3))
        out[i] = np.clip(np.rint(img * 255.0), 0, 255).astype(np.uint8).reshape(-1)
    return out


def make_dataset(cfg: Config, split: str, n: int = None, seed: int = None):
    """Draw ``n`` samples of ``split`` ('train' or 'test') for ``cfg``.

    The draw depends only on (seed, split, n), so a prefix of a larger draw
    is not guaranteed; callers that need a subset slice a full draw.
    """
    if n is None:
        n = cfg.n_train if split == "train" else cfg.n_test
    if seed is None:
        seed = cfg.data_seed
    rng = np.random.default_rng([seed, _GEN_TAGS[split], n])
    priors = cfg.priors if len(cfg.priors) == cfg.n_classes else (1.0,) * cfg.n_classes
    labels = _labels(rng, n, priors)
    if cfg.data_kind == "gauss30":
        values = _gauss30(rng, labels, cfg.n_values)
    elif cfg.data_kind == "uniform":
        values = rng.integers(0, 256, size=(n, cfg.n_values), dtype=np.uint8)
    elif cfg.data_kind == "digits":
        values = _digits(rng, labels, cfg.n_classes, seed)
    elif cfg.data_kind == "lesions":
        values = _lesions(rng, labels, cfg.n_classes, seed)
    else:
        raise ValueError(f"unknown data kind {cfg.data_kind!r}")
    assert values.shape == (n, cfg.n_values)
    return np.ascontiguousarray(values), np.ascontiguousarray(labels)
