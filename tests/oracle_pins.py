"""Pins for the FP64 oracle: facts fixed by the mathematics of the DFT.

Every pin takes an ``OracleLib`` (a compiled copy of ``oracle/oracle.c``) and
raises ``AssertionError`` when that copy disagrees with something other than
itself: hand-evaluated textbook values (``tests/golden``), closed forms
(impulse, shifted impulse, constant, pure tone), theorems (Parseval,
linearity, shift, conjugate symmetry, inversion), brute force against the
O(N^2) definition, and an independent library witness (``torch.fft`` in
complex128 on the CPU).  The same pins are run against copies of the oracle
with planted mistakes to show that each kind of mistake is caught.

Definition pinned (paper Sec. III-A): X[k] = sum_n x[n] exp(sign*2*pi*i*n*k/N),
sign -1 forward, +1 inverse, unnormalised.
"""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "dft_textbook.txt")

POW2 = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]
MIXED = [3, 6, 12, 24, 96, 192, 768, 5, 10, 40, 160, 640, 7, 14, 56, 224, 896, 3072]
PRIMES = [11, 13, 31, 97, 127, 257, 1009]
ALL_N = POW2 + MIXED + PRIMES


def _rng(seed):
    return np.random.default_rng(seed)


def _rand(n, seed, batch=None):
    r = _rng(seed)
    shape = (n,) if batch is None else (batch, n)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _odd_part(n):
    m = n
    while m > 1 and m % 2 == 0:
        m //= 2
    return m


def _roots(n, sign, idx):
    """exp(sign*2*pi*i*idx/n) with idx reduced exactly in integers first."""
    idx = np.asarray(idx, dtype=np.int64) % n
    return np.exp(sign * 2j * np.pi * idx.astype(np.float64) / n)


def _close(a, b, tol, what):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    scale = max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    err = float(np.max(np.abs(a - b))) if a.size else 0.0
    assert err <= tol * scale, f"{what}: max abs err {err:.3e} > {tol:.1e} * {scale:.3g}"


def load_golden(path: str = GOLDEN):
    cases, cur = [], None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "case":
                cur = {"name": vals[0]}
                cases.append(cur)
            elif key in ("n", "sign"):
                cur[key] = int(vals[0])
            elif key in ("x", "X"):
                v = np.array([float(t) for t in vals])
                cur[key] = v[0::2] + 1j * v[1::2]
    for c in cases:
        assert c["x"].shape[0] == c["n"] == c["X"].shape[0], c["name"]
    return cases


# --------------------------------------------------------------------------
# pins
# --------------------------------------------------------------------------
def pin_golden(o):
    """Every routine reproduces the hand-evaluated textbook transforms."""
    for c in load_golden():
        n, s = c["n"], c["sign"]
        _close(o.dft_naive(c["x"], s), c["X"], 1e-14, c["name"] + " naive")
        _close(o.fft(c["x"], s), c["X"], 1e-14, c["name"] + " fft")
        _close(o.dft_bins(c["x"], np.arange(n), s), c["X"], 1e-14, c["name"] + " bins")
        if n & (n - 1) == 0:
            _close(o.fft_radix2(c["x"], s), c["X"], 1e-14, c["name"] + " radix2")
        m = _odd_part(n)
        if m in (3, 5, 7):
            _close(o.fft_split_m(c["x"], m, s), c["X"], 1e-14, c["name"] + " split")


def pin_impulse(o):
    """delta[n] -> all ones, exactly, for every N and both directions."""
    for n in ALL_N:
        x = np.zeros(n, complex)
        x[0] = 1.0
        for s in (-1, 1):
            assert np.array_equal(o.fft(x, s), np.ones(n, complex)), f"impulse fft n={n}"
            assert np.array_equal(o.dft_naive(x, s), np.ones(n, complex)), f"impulse naive n={n}"


def pin_shifted_impulse(o):
    """delta[n-n0] -> W_N^(n0*k) (closed form)."""
    for n in ALL_N:
        n0 = (3 * n) // 7 + (1 if n > 1 else 0)
        n0 %= n
        x = np.zeros(n, complex)
        x[n0] = 1.0
        k = np.arange(n)
        for s in (-1, 1):
            _close(o.fft(x, s), _roots(n, s, n0 * k), 1e-12, f"shifted impulse n={n} s={s}")


def pin_constant(o):
    """constant c -> N*c at k=0 and zero elsewhere."""
    for n in ALL_N:
        c = 0.75 - 0.5j
        y = o.fft(np.full(n, c), -1)
        ref = np.zeros(n, complex)
        ref[0] = n * c
        _close(y, ref, 1e-12, f"constant n={n}")


def pin_tone(o):
    """exp(+2*pi*i*f*n/N) -> N at k=f, zero elsewhere (forward)."""
    for n in ALL_N:
        f = (5 * n) // 11
        x = _roots(n, +1, f * np.arange(n))
        ref = np.zeros(n, complex)
        ref[f] = n
        _close(o.fft(x, -1), ref, 1e-12, f"tone n={n}")
        # and the inverse-sign transform of the conjugate tone
        _close(o.fft(np.conj(x), +1), ref, 1e-12, f"tone inv n={n}")


def pin_parseval(o):
    """sum |X|^2 = N * sum |x|^2."""
    for i, n in enumerate(ALL_N):
        x = _rand(n, 100 + i)
        y = o.fft(x, -1)
        lhs, rhs = np.sum(np.abs(y) ** 2), n * np.sum(np.abs(x) ** 2)
        assert abs(lhs - rhs) <= 1e-12 * rhs, f"parseval n={n}"


def pin_linearity(o):
    """F(a x + b y) = a F(x) + b F(y)."""
    for i, n in enumerate(ALL_N):
        x, z = _rand(n, 200 + i), _rand(n, 300 + i)
        a, b = 0.3 - 1.7j, -2.1 + 0.4j
        _close(o.fft(a * x + b * z, -1), a * o.fft(x, -1) + b * o.fft(z, -1),
               1e-12, f"linearity n={n}")


def pin_shift(o):
    """F(x[n - s])[k] = W_N^(s*k) F(x)[k] (circular shift theorem)."""
    for i, n in enumerate(ALL_N):
        x = _rand(n, 400 + i)
        s = (2 * n) // 5
        k = np.arange(n)
        _close(o.fft(np.roll(x, s), -1), _roots(n, -1, s * k) * o.fft(x, -1),
               1e-12, f"shift n={n}")


def pin_conjugate_symmetry(o):
    """Real input: X[(N-k) mod N] = conj(X[k])."""
    for i, n in enumerate(ALL_N):
        x = _rng(500 + i).standard_normal(n).astype(complex)
        y = o.fft(x, -1)
        _close(y[(-np.arange(n)) % n], np.conj(y), 1e-12, f"hermitian n={n}")


def pin_round_trip(o):
    """inverse(forward(x)) / N = x."""
    for i, n in enumerate(ALL_N):
        x = _rand(n, 600 + i)
        _close(o.fft(o.fft(x, -1), +1) / n, x, 1e-12, f"round trip n={n}")


def pin_brute_force(o):
    """Every fast routine equals the O(N^2) definition."""
    for i, n in enumerate(ALL_N):
        x = _rand(n, 700 + i)
        for s in (-1, 1):
            ref = o.dft_naive(x, s)
            _close(o.fft(x, s), ref, 1e-11, f"fft vs naive n={n}")
            if n & (n - 1) == 0:
                _close(o.fft_radix2(x, s), ref, 1e-11, f"radix2 vs naive n={n}")
            m = _odd_part(n)
            if m in (3, 5, 7):
                _close(o.fft_split_m(x, m, s), ref, 1e-11, f"split vs naive n={n}")
            ks = np.array([0, 1, n // 2, n - 1, (7 * n) // 9])
            _close(o.dft_bins(x, ks, s), ref[ks % n], 1e-11, f"bins n={n}")


def pin_batch(o):
    """Batched transform = each row transformed alone (threads over the batch)."""
    x = _rand(192, 800, batch=9)
    y = o.fft(x, -1, threads=4)
    for b in range(9):
        _close(y[b], o.dft_naive(x[b], -1), 1e-11, f"batch row {b}")


def pin_library_witness(o):
    """Independent witness: torch.fft.fft (pocketfft) in complex128 on the CPU."""
    import torch
    for i, n in enumerate(ALL_N + [65536, 3 * 16384, 4099]):
        x = _rand(n, 900 + i)
        t = torch.from_numpy(x)
        _close(o.fft(x, -1), torch.fft.fft(t).numpy(), 1e-11, f"torch fwd n={n}")
        _close(o.fft(x, +1), (torch.fft.ifft(t) * n).numpy(), 1e-11, f"torch inv n={n}")


def pin_2d(o):
    """2-D: brute-force double sum on tiny shapes, separability, library witness."""
    import torch
    for (h, w) in [(1, 1), (2, 3), (4, 6), (8, 5), (3, 16)]:
        x = _rand(h * w, 1000 + h * 31 + w).reshape(h, w)
        k1 = np.arange(h)[:, None, None, None]
        k2 = np.arange(w)[None, :, None, None]
        n1 = np.arange(h)[None, None, :, None]
        n2 = np.arange(w)[None, None, None, :]
        for s in (-1, 1):
            ph = _roots(h, s, k1 * n1) * _roots(w, s, k2 * n2)
            ref = np.sum(ph * x[None, None], axis=(2, 3))
            _close(o.fft2(x, s), ref, 1e-12, f"2d brute {h}x{w}")
    x = _rand(2 * 32 * 64, 1100).reshape(2, 32, 64)
    _close(o.fft2(x, -1), torch.fft.fft2(torch.from_numpy(x)).numpy(), 1e-11, "2d torch")


def pin_image_dc_and_spikes(o):
    """Image-shaped data: X[0,0] is the exact integer sum (the integer-period
    sinusoid sums to zero) and the sinusoid puts spikes of H*W*amp/2 at
    (+-fy, +-fx) on top of the integer part's spectrum."""
    r = _rng(1200)
    h, w, amp, fx, fy = 32, 64, 32.0, 3, 2
    ints = r.integers(0, 256, (h, w))
    yy, xx = np.mgrid[0:h, 0:w]
    field = amp * np.sin(2 * np.pi * (fx * xx / w + fy * yy / h))
    X = o.fft2((ints + field).astype(complex), -1)
    assert abs(X[0, 0] - int(ints.sum())) <= 1e-9 * h * w * 255, "DC"
    Xi = o.fft2(ints.astype(complex), -1)
    spike = h * w * amp / 2
    _close(X[fy, fx] - Xi[fy, fx], -1j * spike, 1e-9, "spike +")
    _close(X[-fy % h, -fx % w] - Xi[-fy % h, -fx % w], 1j * spike, 1e-9, "spike -")


def pin_convolution(o):
    """Circular convolution / correlation: impulse kernel is the identity, a
    shifted impulse shifts (conv) or shifts back (corr), a constant kernel
    sums, hand-evaluated 4-point case, commutativity, and the convolution
    theorem against the torch.fft witness."""
    import torch
    for i, n in enumerate([1, 2, 3, 7, 16, 30, 97]):
        x = _rand(n, 1300 + i)
        d = np.zeros(n, complex)
        d[0] = 1
        _close(o.circ_conv(x, d), x, 1e-13, f"conv identity n={n}")
        _close(o.circ_conv(x, d, corr=True), x, 1e-13, f"corr identity n={n}")
        s = (3 * n) // 5
        ds = np.zeros(n, complex)
        ds[s] = 1
        _close(o.circ_conv(x, ds), np.roll(x, s), 1e-13, f"conv shift n={n}")
        _close(o.circ_conv(x, ds, corr=True), np.roll(x, -s), 1e-13, f"corr shift n={n}")
        c = np.full(n, 0.5 - 0.25j)
        _close(o.circ_conv(x, c), np.full(n, (0.5 - 0.25j) * x.sum()), 1e-12, f"conv constant n={n}")
        h = _rand(n, 1400 + i)
        _close(o.circ_conv(x, h), o.circ_conv(h, x), 1e-12, f"conv commutes n={n}")
        tx, th = torch.from_numpy(x), torch.from_numpy(h)
        conv = torch.fft.ifft(torch.fft.fft(tx) * torch.fft.fft(th)).numpy()
        corr = torch.fft.ifft(torch.fft.fft(tx) * torch.fft.fft(th).conj()).numpy()
        _close(o.circ_conv(x, h), conv, 1e-11, f"conv theorem n={n}")
        _close(o.circ_conv(x, h, corr=True), corr, 1e-11, f"corr theorem n={n}")
    # [1,2,3,4] (*) [1,1,0,0]: y[m] = x[m] + x[m-1] = [5, 3, 5, 7]
    _close(o.circ_conv(np.array([1, 2, 3, 4], complex), np.array([1, 1, 0, 0], complex)),
           np.array([5, 3, 5, 7], complex), 1e-14, "conv 4-point")


# --------------------------------------------------------------------------
# image example (Sec. III-B) steps 1-3: colour transform, chroma 2x2 mean,
# directional derivative of luminance
# --------------------------------------------------------------------------
def _rgb(b, h, w, seed):
    return _rng(seed).integers(0, 256, (b, h, w, 3)).astype(np.uint8)


def pin_ycc_gray(o):
    """Gray pixels (R = G = B = v) have Y = v and no colour: Cb = Cr = 128."""
    v = np.arange(0, 256, 5, dtype=np.uint8)
    rgb = np.repeat(np.repeat(v[:, None, None, None], 4, 1), 6, 2).repeat(3, 3)
    y, cb, cr, _ = o.image_steps(rgb)
    _close(y, np.broadcast_to(v[:, None, None].astype(float), y.shape), 1e-12, "gray luma")
    _close(cb, np.full(cb.shape, 128.0), 1e-12, "gray Cb")
    _close(cr, np.full(cr.shape, 128.0), 1e-12, "gray Cr")


def pin_ycc_inverse(o):
    """The published JFIF inverse (R = Y + 1.402 (Cr-128), G = Y - 0.344136
    (Cb-128) - 0.714136 (Cr-128), B = Y + 1.772 (Cb-128)) recovers every colour
    (constant 2x2 images, so the downscaled chroma is the pixel's chroma)."""
    cols = _rgb(1, 1, 300, 40)[0, 0]
    rgb = np.repeat(np.repeat(cols[:, None, None, :], 2, 1), 2, 2)
    y, cb, cr, _ = o.image_steps(rgb)
    Y, Cb, Cr = y[:, 0, 0], cb[:, 0, 0] - 128.0, cr[:, 0, 0] - 128.0
    back = np.stack([Y + 1.402 * Cr, Y - 0.344136 * Cb - 0.714136 * Cr, Y + 1.772 * Cb], 1)
    err = float(np.max(np.abs(back - cols.astype(float))))
    assert err <= 2e-3, f"JFIF inverse misses the colour by {err:.3e}"


def pin_ycc_colour_difference(o):
    """BT.601 colour differences: Cb - 128 = (B - Y) / (2 (1 - 0.114)) and
    Cr - 128 = (R - Y) / (2 (1 - 0.299))."""
    cols = _rgb(1, 1, 200, 41)[0, 0].astype(np.uint8)
    rgb = np.repeat(np.repeat(cols[:, None, None, :], 2, 1), 2, 2)
    y, cb, cr, _ = o.image_steps(rgb)
    Y = y[:, 0, 0]
    R, B = cols[:, 0].astype(float), cols[:, 2].astype(float)
    assert float(np.max(np.abs(cb[:, 0, 0] - 128.0 - (B - Y) / 1.772))) <= 2e-3, "Cb colour difference"
    assert float(np.max(np.abs(cr[:, 0, 0] - 128.0 - (R - Y) / 1.402))) <= 2e-3, "Cr colour difference"


def pin_chroma_block_mean(o):
    """Downscaled chroma = mean over each 2x2 block of the chroma of its four
    pixel colours (each taken from a constant 2x2 image)."""
    rgb = _rgb(2, 6, 8, 42)
    _, cb, cr, _ = o.image_steps(rgb)
    for b in range(2):
        for j in range(3):
            for i in range(4):
                px = rgb[b, 2 * j:2 * j + 2, 2 * i:2 * i + 2].reshape(4, 3)
                one = np.repeat(np.repeat(px[:, None, None, :], 2, 1), 2, 2)
                _, cbs, crs, _ = o.image_steps(one)
                assert abs(cb[b, j, i] - cbs.mean()) <= 1e-9, ("Cb block", b, j, i)
                assert abs(cr[b, j, i] - crs.mean()) <= 1e-9, ("Cr block", b, j, i)


def pin_derivative_closed_forms(o):
    """Gray ramps: Y = a x + b y + c has directional derivative ux a + uy b
    everywhere (central differences inside, one-sided on the border, both
    exact for a linear function); Y = x^2 has 2x inside, 1 and 2w - 3 on the
    left and right borders; a constant has 0."""
    h, w = 6, 10
    yy, xx = np.mgrid[0:h, 0:w]
    for a, bb, c, ux, uy in ((3, 7, 11, 1.0, 0.0), (3, 7, 11, 0.0, 1.0), (5, 2, 9, 0.6, 0.8),
                             (-4, 9, 200, -0.8, 0.6)):
        g = (a * xx + bb * yy + c).astype(np.uint8)
        rgb = np.repeat(g[None, :, :, None], 3, 3)
        y, _, _, d = o.image_steps(rgb, ux, uy)
        _close(y[0], g.astype(float), 1e-12, "ramp luma")
        _close(d[0], np.full((h, w), ux * a + uy * bb), 1e-12, f"ramp derivative {(a, bb, ux, uy)}")
    g = (xx ** 2).astype(np.uint8)
    _, _, _, d = o.image_steps(np.repeat(g[None, :, :, None], 3, 3), 1.0, 0.0)
    want = 2.0 * xx.astype(float)
    want[:, 0] = 1.0
    want[:, w - 1] = 2 * w - 3
    _close(d[0], want, 1e-12, "quadratic derivative")
    _, _, _, d = o.image_steps(np.full((1, 4, 4, 3), 77, np.uint8), 0.6, 0.8)
    _close(d, np.zeros_like(d), 1e-12, "constant derivative")


def pin_derivative_linear_in_direction(o):
    """D(ux, uy) = ux D(1, 0) + uy D(0, 1) on random images."""
    rgb = _rgb(2, 8, 12, 43)
    _, _, _, dx = o.image_steps(rgb, 1.0, 0.0)
    _, _, _, dy = o.image_steps(rgb, 0.0, 1.0)
    _, _, _, du = o.image_steps(rgb, 0.28, -0.96)
    _close(du, 0.28 * dx - 0.96 * dy, 1e-12, "derivative linearity")


ALL_PINS = [pin_golden, pin_impulse, pin_shifted_impulse, pin_constant, pin_tone,
            pin_parseval, pin_linearity, pin_shift, pin_conjugate_symmetry,
            pin_round_trip, pin_brute_force, pin_batch, pin_library_witness,
            pin_2d, pin_image_dc_and_spikes, pin_convolution,
            pin_ycc_gray, pin_ycc_inverse, pin_ycc_colour_difference, pin_chroma_block_mean,
            pin_derivative_closed_forms, pin_derivative_linear_in_direction]


def failing_pins(o):
    """Names of pins that reject oracle copy ``o``."""
    bad = []
    for p in ALL_PINS:
        try:
            p(o)
        except AssertionError:
            bad.append(p.__name__)
    return bad
