"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here retypes the oracle's update formulas: the temporal filter is checked
against the transfer functions of Eqs. 12-14 run through scipy's LTI filter, against
Eq. 15 (the paper's single second-order recurrence), against periodic steady states
computed in the frequency domain and against closed forms; the detector against an
independent brute-force recount and hand-worked traces (tests/golden); the blur
against scipy's convolution.
"""
import math
import os

import numpy as np
import pytest
import torch
from scipy import ndimage, signal

import eventsim
from tests import bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def prefix_trick_events(train, W):
    """Pixel i (0 <= i < len(train)) receives the first i+1 polarities of ``train``.

    After one read-out, pixel i holds the filter state after i+1 events, so a single
    read-out returns the whole response sequence.  Spatial filtering is off (NSF) so
    pixels cannot influence one another.
    """
    n = len(train)
    xs, ys, ps = [], [], []
    for step in range(n):
        for i in range(step, n):       # all pixels that still need event `step`
            xs.append(i % W)
            ys.append(i // W)
            ps.append(train[step])
    t = np.arange(len(xs))
    return eventsim.pack_events(torch.tensor(xs), torch.tensor(ys), torch.tensor(ps),
                                torch.from_numpy(t))


def run_train(oracle_mod, train, t_cut=40.0, c_on=1.0, c_off=1.0):
    n = len(train)
    W = n
    o = oracle_mod.Oracle(W, 1, t_cut=t_cut, c_on=c_on, c_off=c_off, spatial_filter=0)
    o.push(prefix_trick_events(train, W))
    img = o.readout(2**62)
    return img.reshape(-1)[:n], o


# --- coefficients (Eqs. 16-18) -----------------------------------------------------

def H_alpha(z, a):
    return a * (z - 1) / (z - a)          # Eq. 13


def H_beta(z, b):
    return z * (1 + b) / (2 * (z - b))    # Eq. 14


@pytest.mark.parametrize("t_cut", [7.0, 40.0, 100.0, 1000.0])
def test_coefficients_half_power(oracle_mod, t_cut):
    """alpha and beta put the half-power point of H_alpha (high pass, maximum at
    omega = pi) and H_beta (low pass, maximum at omega = 0) at omega_cut = 2 pi / T_cut
    (Sec. 4.1, the text around Eqs. 17-18)."""
    a, b = oracle_mod.coefficients(t_cut)
    w = 2 * math.pi / t_cut
    z = np.exp(1j * w)
    ra = abs(H_alpha(z, a)) ** 2 / abs(H_alpha(-1.0, a)) ** 2
    rb = abs(H_beta(z, b)) ** 2 / abs(H_beta(1.0, b)) ** 2
    # Eq. 18 subtracts two nearly equal numbers when omega_cut is small: its rounding
    # error grows like eps / omega_cut
    tol = 1e-13 * t_cut
    assert ra == pytest.approx(0.5, abs=tol)
    assert rb == pytest.approx(0.5, abs=tol)
    # H_alpha is maximal at omega = pi, H_beta at omega = 0
    grid = np.exp(1j * np.linspace(0, math.pi, 2001))
    assert np.argmax(abs(H_alpha(grid, a))) == 2000
    assert np.argmax(abs(H_beta(grid, b))) == 0
    assert 0 < a < 1 and 0 < b < 1


def test_coefficients_taylor_and_known_values(oracle_mod):
    """Both coefficients agree with 1 - w + w^2/2 to O(w^3) (Sec. 4.1)."""
    for t_cut in [200.0, 400.0, 800.0]:
        a, b = oracle_mod.coefficients(t_cut)
        w = 2 * math.pi / t_cut
        taylor = 1 - w + w * w / 2
        assert abs(a - taylor) < 2 * w ** 3
        assert abs(b - taylor) < 2 * w ** 3
    a, b = oracle_mod.coefficients(float("inf"))
    assert a == 1.0 and b == 1.0


# --- temporal filter ---------------------------------------------------------------

def lti_response(train_scaled, a, b):
    """H(z) = H_alpha H_beta = (a(1+b)/2) (1 - z^-1) / ((1 - a z^-1)(1 - b z^-1))."""
    g = a * (1 + b) / 2
    return signal.lfilter([g, -g], [1.0, -(a + b), a * b], train_scaled)


@pytest.mark.parametrize("t_cut,c_on,c_off,seed", [(40.0, 1.0, 1.0, 0), (100.0, 1.0, 1.0, 1),
                                                    (40.0, 0.2, 0.3, 2), (12.0, 0.7, 0.25, 3)])
def test_iir_matches_transfer_function(oracle_mod, t_cut, c_on, c_off, seed):
    """The per-event filter of Eqs. 6, 7, 10 realises H(z) = H_alpha(z) H_beta(z)
    (Eqs. 12-14) applied to the increments C_p p (Eq. 3)."""
    rng = np.random.default_rng(seed)
    train = list(np.where(rng.random(60) < 0.45, 1, -1))
    L, o = run_train(oracle_mod, train, t_cut, c_on, c_off)
    # the contrast scales are float32 parameters
    con, coff = float(np.float32(c_on)), float(np.float32(c_off))
    scaled = np.array([con if p > 0 else -coff for p in train])
    ref = lti_response(scaled, o.alpha, o.beta)
    np.testing.assert_allclose(L, ref, rtol=0, atol=1e-12)


def test_iir_matches_eq15(oracle_mod):
    """Eq. 15, the single second-order recurrence, gives the same output."""
    rng = np.random.default_rng(7)
    train = list(np.where(rng.random(50) < 0.6, 1, -1))
    L, o = run_train(oracle_mod, train, 40.0)
    a, b = o.alpha, o.beta
    y = []
    y1 = y2 = 0.0
    p1 = 0.0
    for p in train:
        yk = (a + b) * y1 - a * b * y2 + 0.5 * a * (1 + b) * (p - p1)
        y.append(yk)
        y2, y1, p1 = y1, yk, p
    np.testing.assert_allclose(L, y, rtol=0, atol=1e-12)


def test_iir_hand_computed_trains(oracle_mod):
    """Closed forms worked by hand from Eqs. 6, 7, 10 with zero initial state:
    [+1] -> g a ; [+1,+1] -> g a (a + b) ; [+1,-1] -> g(-a(1+a) + a b) ... with
    g = (1+b)/2."""
    a, b = oracle_mod.coefficients(40.0)
    g = (1 + b) / 2
    L, _ = run_train(oracle_mod, [1, 1, -1], 40.0)
    assert L[0] == pytest.approx(g * a, abs=1e-14)
    assert L[1] == pytest.approx(g * a * (a + b), abs=1e-14)
    # third event -1: pbar_2 = (1-a)(1+a); pbar_3 = a pbar_2 - (1-a); dL = -1 - pbar_3
    pbar3 = a * (1 - a) * (1 + a) - (1 - a)
    assert L[2] == pytest.approx(b * L[1] + g * (-1 - pbar3), abs=1e-14)
    assert g * a == pytest.approx(0.7921219265955229, abs=1e-13)
    L2, _ = run_train(oracle_mod, [1, -1], 40.0)
    assert L2[1] == pytest.approx(-0.2305138860630270, abs=1e-13)


def test_iir_steady_states(oracle_mod):
    """DC rejection (H(1) = 0) and the Nyquist gain H(-1) = a / (1 + a)."""
    L, o = run_train(oracle_mod, [1] * 400, 40.0)
    assert abs(L[-1]) < 1e-12
    alt = [1 if i % 2 == 0 else -1 for i in range(400)]
    L, o = run_train(oracle_mod, alt, 40.0)
    gain = o.alpha / (1 + o.alpha)
    assert abs(abs(L[-1]) - gain) < 1e-12
    assert L[-1] * alt[-1] > 0
    assert gain == pytest.approx(0.4606491465876907, abs=1e-13)


@pytest.mark.parametrize("n_on,n_off", [(5, 5), (3, 7), (10, 10)])
def test_iir_periodic_steady_state_frequency_domain(oracle_mod, n_on, n_off):
    """A periodic train ON^n_on OFF^n_off settles to the periodic response given by
    H(e^{j 2 pi m / P}) on its Fourier coefficients (Fig. 2's transfer function)."""
    P = n_on + n_off
    period = np.array([1.0] * n_on + [-1.0] * n_off)
    reps = 60
    train = list(np.tile(period, reps).astype(int))
    L, o = run_train(oracle_mod, train, 40.0)
    a, b = o.alpha, o.beta
    z = np.exp(2j * math.pi * np.arange(P) / P)
    with np.errstate(divide="ignore", invalid="ignore"):
        H = H_alpha(z, a) * H_beta(z, b)
    H[0] = 0.0  # H(1) = 0
    y_ss = np.real(np.fft.ifft(np.fft.fft(period) * H))
    np.testing.assert_allclose(L[-P:], y_ss, rtol=0, atol=1e-9)


def test_alpha_beta_one_is_simple_sum(oracle_mod):
    """alpha = beta = 1 (T_cut -> infinity) reduces FIBAR to Eq. 4/5: L = sum C_p p."""
    rng = np.random.default_rng(3)
    train = list(np.where(rng.random(80) < 0.5, 1, -1))
    L, _ = run_train(oracle_mod, train, float("inf"), c_on=0.5, c_off=0.25)
    ref = np.cumsum([0.5 if p > 0 else -0.25 for p in train])
    np.testing.assert_array_equal(L, ref)


# --- detector (Sec. 4.2, Eqs. 19-20) -------------------------------------------------

def _load_golden():
    cases = {}
    cur = None
    with open(os.path.join(GOLDEN, "detector_2x2.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("case"):
                parts = line.split()
                kv = dict(p.split("=") for p in parts[2:])
                cur = dict(q_min=int(kv["q_min"]), q_init=int(kv["q_init"]), rows=[])
                cases[parts[1]] = cur
                continue
            a, b, c = line.split("|")
            k, pix = map(int, a.split())
            h, qt, nap, nat = map(int, b.split())
            stale = [int(s) for s in c.split()]
            cur["rows"].append((k, pix, h, qt, nap, nat, stale))
    return cases


@pytest.mark.parametrize("case", ["cycle", "repeat", "pair"])
def test_detector_hand_worked(oracle_mod, case):
    c = _load_golden()[case]
    pix = [r[1] for r in c["rows"]]
    ev = eventsim.pack_events(torch.tensor([p % 2 for p in pix]), torch.tensor([p // 2 for p in pix]),
                              torch.ones(len(pix), dtype=torch.int64), torch.arange(len(pix)))
    o = oracle_mod.Oracle(2, 2, q_min=c["q_min"], q_init=c["q_init"])
    o.start_trace(64)
    o.push(ev)
    o.flush()
    tr = o.trace()
    bf = bruteforce.detector_trace(2, 2, pix, q_min=c["q_min"], q_init=c["q_init"])
    for i, (k, p, h, qt, nap, nat, stale) in enumerate(c["rows"]):
        assert tr["h"][i] == h and bf["h"][i] == h
        assert tr["q_targ"][i] == qt and bf["q_targ"][i] == qt
        assert tr["n_ap"][i] == nap and bf["n_ap"][i] == nap
        assert tr["n_at"][i] == nat and bf["n_at"][i] == nat
        got = [int(px) for kk, px in zip(tr["stale_k"], tr["stale_pix"]) if kk == k]
        assert got == stale
        assert [px for kk, px in bf["stale"] if kk == k] == stale


def _stream_cases():
    yield "random4x4", 4, 4, eventsim.random_events(4, 4, 400, seed=1), dict(q_min=1)
    yield "random6x4", 6, 4, eventsim.random_events(6, 4, 500, seed=2), dict(q_min=2, q_init=3)
    yield "random8x8", 8, 8, eventsim.random_events(8, 8, 800, seed=3), dict(q_min=1)
    yield "onetile8x8", 8, 8, eventsim.random_events(8, 8, 300, seed=4, pixels=[18, 19, 26, 27]), dict(q_min=1)
    yield "onepixel", 4, 4, eventsim.random_events(4, 4, 100, seed=5, pixels=[5]), dict(q_min=1)
    yield "odd5x3", 5, 3, eventsim.random_events(5, 3, 300, seed=6), dict(q_min=1)
    yield "fill07", 8, 8, eventsim.random_events(8, 8, 600, seed=7), dict(q_min=1, fill_num=7, fill_den=10)
    ev = eventsim.simulate(16, 12, 3000, scene=eventsim.SceneSpec(texture="sine_checker", cell_px=4,
                                                                   period_px=6.0), seed=8)
    yield "edge16x12", 16, 12, ev, dict()


@pytest.mark.parametrize("name,W,H,ev,kw", list(_stream_cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_detector_matches_bruteforce(oracle_mod, name, W, H, ev, kw):
    """Per-event window, counts, q_targ and the ordered stale list equal a from-scratch
    recount at every step."""
    x, y, p, t = eventsim.unpack_events(ev)
    pix = (y * W + x).tolist()
    o = oracle_mod.Oracle(W, H, **kw)
    o.start_trace(len(pix))
    o.push(ev)
    o.flush()
    tr = o.trace()
    bf = bruteforce.detector_trace(W, H, pix, **{k: v for k, v in kw.items()})
    np.testing.assert_array_equal(tr["h"], bf["h"])
    np.testing.assert_array_equal(tr["q_targ"], bf["q_targ"])
    np.testing.assert_array_equal(tr["n_ap"], bf["n_ap"])
    np.testing.assert_array_equal(tr["n_at"], bf["n_at"])
    assert tr["n_stale"] == len(bf["stale"])
    assert list(zip(tr["stale_k"].tolist(), tr["stale_pix"].tolist())) == bf["stale"]


def test_detector_invariants(oracle_mod):
    """Invariants of the window: sum cnt = q, sum tcnt = N_ap, N_at <= N_ap <= min(q, 4 N_at)
    (fill ratio in [1/4, 1], Eq. 19), q_min <= q_targ <= q_max, stale = ever & cnt == 0."""
    W, H = 24, 18
    ev = eventsim.simulate(W, H, 20000, scene="sine_checker", seed=3, noise_frac=0.05)
    o = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2)
    step = 997
    hs = []
    for i in range(0, 20000, step):
        o.push(ev[i:i + step])
        o.flush()
        s = o.state()
        q = s["q"]
        assert int(s["cnt"].sum()) == q
        assert int(s["tcnt"].sum()) == s["n_ap"]
        assert s["n_at"] <= s["n_ap"] <= min(q, 4 * s["n_at"])
        assert o.q_min <= s["q_targ"] <= o.q_max
        assert q == s["k"] - s["h"]
        hs.append(s["h"])
        # tile counts are the number of active pixels per 2x2 tile
        act = (s["cnt"] > 0).reshape(H, W)
        tc = act.reshape(H // 2, 2, W // 2, 2).sum(axis=(1, 3)).reshape(-1)
        np.testing.assert_array_equal(tc, s["tcnt"])
    assert hs == sorted(hs)


def test_detector_closed_form_trajectories(oracle_mod):
    """Closed forms: one pixel firing -> N_ap = N_at = 1, q_targ = min(2q, W H), the queue
    grows by one per event and nothing goes stale; four pixels of one tile in turn ->
    fixed point r = 1/2 at q = 2 with one stale pixel per event; pixels in distinct
    tiles -> r = 1/4, the target doubles."""
    W, H = 8, 8
    ev = eventsim.random_events(W, H, 100, seed=0, pixels=[9])
    o = oracle_mod.Oracle(W, H, q_min=1)
    o.start_trace(100)
    o.push(ev)
    o.flush()
    tr = o.trace()
    q = np.arange(1, 101)
    qk = np.minimum(q, 64)
    np.testing.assert_array_equal(tr["h"], np.arange(100) + 1 - qk)
    np.testing.assert_array_equal(tr["q_targ"], np.minimum(2 * qk, 64))
    assert tr["n_stale"] == 0
    # one tile, pixels visited in turn
    tile = [0, 1, 8, 9]
    pix = [tile[i % 4] for i in range(200)]
    ev = eventsim.pack_events(torch.tensor([p % W for p in pix]), torch.tensor([p // W for p in pix]),
                              torch.ones(200, dtype=torch.int64), torch.arange(200))
    o = oracle_mod.Oracle(W, H, q_min=1)
    o.start_trace(200)
    o.push(ev)
    o.flush()
    tr = o.trace()
    k = np.arange(200)
    assert np.all(k[20:] + 1 - tr["h"][20:] == 2)
    assert np.all(tr["n_ap"][20:] == 2) and np.all(tr["n_at"][20:] == 1)
    st = dict(zip(tr["stale_k"].tolist(), tr["stale_pix"].tolist()))
    for kk in range(20, 200):
        assert st[kk] == pix[kk - 2]
    # the same cycle with q_min = 3: the fixed point q = 2 lies below the bound, so the
    # queue is held at 3 and the pixel of event k-3 goes stale at step k
    o = oracle_mod.Oracle(W, H, q_min=3)
    o.start_trace(200)
    o.push(ev)
    o.flush()
    tr = o.trace()
    assert np.all(k[20:] + 1 - tr["h"][20:] == 3)
    assert np.all(tr["q_targ"][20:] == 3)
    st = dict(zip(tr["stale_k"].tolist(), tr["stale_pix"].tolist()))
    for kk in range(20, 200):
        assert st[kk] == pix[kk - 3]
    # distinct tiles: the target doubles each event (until the cap)
    pix = [0, 2, 4, 6, 16, 18, 20, 22]
    ev = eventsim.pack_events(torch.tensor([p % W for p in pix]), torch.tensor([p // W for p in pix]),
                              torch.ones(8, dtype=torch.int64), torch.arange(8))
    o = oracle_mod.Oracle(W, H, q_min=1)
    o.start_trace(8)
    o.push(ev)
    o.flush()
    tr = o.trace()
    np.testing.assert_array_equal(tr["q_targ"], np.minimum(2 * np.arange(1, 9), 64))
    np.testing.assert_array_equal(tr["n_ap"], tr["n_at"])


# --- blur (Sec. 4.2: one-time 3x3 Gaussian) ---------------------------------------------

def scipy_blur(img):
    k = np.outer([1.0, 2.0, 1.0], [1.0, 2.0, 1.0])
    num = ndimage.convolve(img, k, mode="constant", cval=0.0)
    den = ndimage.convolve(np.ones_like(img), k, mode="constant", cval=0.0)
    return num / den


def test_blur_matches_renormalised_convolution(oracle_mod):
    rng = np.random.default_rng(0)
    for H, W in [(8, 8), (5, 7), (1, 6), (6, 1), (1, 1), (2, 3)]:
        img = rng.normal(size=(H, W))
        np.testing.assert_allclose(oracle_mod.blur_image(img), scipy_blur(img), atol=1e-13)
    const = np.full((6, 9), 0.37)
    np.testing.assert_allclose(oracle_mod.blur_image(const), const, atol=1e-15)
    imp = np.zeros((8, 8))
    imp[0, 0] = 1.0
    b = oracle_mod.blur_image(imp)
    assert b[0, 0] == pytest.approx(4 / 9) and b[0, 1] == pytest.approx(2 / 12)
    assert b[1, 1] == pytest.approx(1 / 16)


# --- whole-pipeline behaviour ------------------------------------------------------------

def test_untouched_pixels_stay_zero(oracle_mod):
    """A pixel without events keeps its value (Sec. 4.1); in S1 it is never blurred
    because it never enters the queue."""
    W, H = 32, 24
    ev = eventsim.simulate(W, H, 5000, scene="sine_checker", seed=2)
    x, y, p, t = eventsim.unpack_events(ev)
    keep = (x < 20)
    ev = ev[keep]
    for mode in [dict(spatial_filter=0), dict(blur_mode=0), dict(blur_mode=1)]:
        o = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2, **mode)
        o.push(ev)
        o.flush()
        s = o.state()
        L = s["L"].reshape(H, W)
        assert np.all(L[:, 20:] == 0.0)
        assert np.all(s["pbar"].reshape(H, W)[:, 20:] == 0.0)


def test_nsf_pixels_are_independent(oracle_mod):
    """Without spatial filtering every pixel is its own filter: a stream restricted to
    one pixel gives that pixel the same value as in the full stream."""
    W, H = 16, 12
    ev = eventsim.simulate(W, H, 4000, scene="sine_checker", seed=4)
    x, y, p, t = eventsim.unpack_events(ev)
    o = oracle_mod.Oracle(W, H, spatial_filter=0)
    o.push(ev)
    full = o.readout(2**62)
    for pix in [0, 37, 100, W * H - 1]:
        sel = (y * W + x) == pix
        o2 = oracle_mod.Oracle(W, H, spatial_filter=0)
        o2.push(ev[sel])
        one = o2.readout(2**62)
        assert one.reshape(-1)[pix] == full.reshape(-1)[pix]


def test_s2_readout_is_masked_blur_of_state(oracle_mod):
    """S2 read-out = blur(L) where the pixel is stale (had an event, none queued),
    L elsewhere; the state itself is never blurred."""
    W, H = 20, 16
    ev = eventsim.simulate(W, H, 6000, scene="sine_checker", seed=5)
    o = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2, blur_mode=1)
    o.push(ev)
    img = o.readout(2**62)
    s = o.state()
    L = s["L"].reshape(H, W)
    stale = ((s["ever"] == 1) & (s["cnt"] == 0)).reshape(H, W)
    assert stale.any() and (~stale).any()
    ref = np.where(stale, scipy_blur(L), L)
    np.testing.assert_allclose(img, ref, atol=1e-13)
    o2 = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2, spatial_filter=0)
    o2.push(ev)
    np.testing.assert_array_equal(o2.readout(2**62), L)   # S2 never changes the state


def test_s1_blur_reads_neighbours_at_that_step(oracle_mod):
    """S1: when the only event of a pixel leaves the queue, its L becomes the blur of
    the current neighbourhood, and later events start from that value (Sec. 4.2)."""
    # 4x2 sensor, q_min = q_init = 1. Events: A=(0,0)+, B=(2,0)+, C=(3,1)-, ...
    # trace the oracle and check every stale step against scipy on the state
    W, H = 6, 4
    ev = eventsim.random_events(W, H, 60, seed=11)
    x, y, p, t = eventsim.unpack_events(ev)
    o = oracle_mod.Oracle(W, H, q_min=1, q_init=1)
    o_nsf = None
    o.start_trace(60)
    for i in range(60):
        before = o.state()
        o.push(ev[i:i + 1])
        o.flush()
        after = o.state()
        tr = o.trace()
        stale_now = [int(px) for kk, px in zip(tr["stale_k"], tr["stale_pix"]) if kk == i]
        pix = int(y[i] * W + x[i])
        # replay the step: IIR of the event, then blurs in pop order
        L = before["L"].copy()
        pb = before["pbar"].copy()
        s_ = 1.0 if p[i] > 0 else -1.0
        pb[pix] = o.alpha * pb[pix] + (1 - o.alpha) * s_
        L[pix] = o.beta * L[pix] + 0.5 * (1 + o.beta) * (s_ - pb[pix])
        for sp in stale_now:
            L[sp] = scipy_blur(L.reshape(H, W)).reshape(-1)[sp]
        np.testing.assert_allclose(after["L"], L, atol=1e-13)
        np.testing.assert_array_equal(after["pbar"], pb)


def test_readout_prefix_and_order(oracle_mod):
    """Read-out at t applies the longest pushed prefix with t_k <= t (Eq. 4's t_k <= t);
    events stay queued until a later read-out; decreasing read-out times are refused."""
    W, H = 10, 8
    ev = eventsim.random_events(W, H, 500, seed=9, t_step_us=10)
    o = oracle_mod.Oracle(W, H)
    o.push(ev)
    o.readout(1234)
    assert o.state()["k"] == 124            # events with t = 0, 10, ..., 1230
    assert o.state()["pending"] == 376
    o.readout(1240)                          # an event exactly at t is applied
    assert o.state()["k"] == 125
    assert o.readout_rc(1000) == -3
    o.readout(1240)
    assert o.state()["k"] == 125
    # non-monotone time stamps: the prefix stops at the first later event
    ev2 = ev.clone()
    ev2[130, 1] = 10**9
    o2 = oracle_mod.Oracle(W, H)
    o2.push(ev2)
    o2.readout(1500)
    assert o2.state()["k"] == 130


def test_packet_split_invariance(oracle_mod):
    W, H = 24, 18
    ev = eventsim.simulate(W, H, 8000, scene="sine_checker", seed=1, noise_frac=0.02)
    ref = None
    for split in [1, 7, 1000, 8000]:
        o = oracle_mod.Oracle(W, H, c_on=0.2, c_off=0.2)
        for i in range(0, 8000, split):
            o.push(ev[i:i + split])
        img = o.readout(2**62)
        s = o.state()
        key = (img.tobytes(), s["cnt"].tobytes(), s["h"], s["q_targ"])
        if ref is None:
            ref = key
        assert key == ref


def test_out_of_range_events_are_dropped(oracle_mod):
    W, H = 8, 6
    ev = eventsim.random_events(W, H, 100, seed=2)
    bad = eventsim.pack_events(torch.tensor([8, 0, 100]), torch.tensor([0, 6, 100]),
                               torch.tensor([1, -1, 1]), torch.tensor([5, 5, 5]))
    mixed = torch.cat([ev[:5], bad, ev[5:]])
    mixed[:, 1] = torch.arange(mixed.shape[0])
    o = oracle_mod.Oracle(W, H)
    o.push(mixed)
    img = o.readout(2**62)
    s = o.state()
    assert s["dropped"] == 3 and s["k"] == 100
    o2 = oracle_mod.Oracle(W, H)
    e2 = ev.clone()
    e2[:, 1] = torch.arange(100)
    o2.push(e2)
    np.testing.assert_array_equal(o2.readout(2**62), img)


def test_invalid_params_rejected(oracle_mod):
    for kw in [dict(t_cut=3.0), dict(fill_num=0), dict(fill_den=0), dict(c_on=0.0),
               dict(blur_mode=2), dict(q_min=100), dict(q_init=2, q_min=3)]:
        with pytest.raises(ValueError):
            oracle_mod.Oracle(8, 8, **kw)
    with pytest.raises(ValueError):
        oracle_mod.Oracle(0, 8)
