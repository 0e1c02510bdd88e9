"""Pins for the oracle's Balloon-Windkessel BOLD and phFCD (oracle/bold.py):
the resting state is a fixed point with zero BOLD; a constant drive settles on
the closed-form fixed point; small drives respond linearly; a brief pulse
gives the hemodynamic response peaking a few seconds later (the published
behaviour of the model); the band-limited analytic signal of an in-band
sinusoid is its complex exponential; phFCD is 1 for phase-locked regions and
matches a brute-force computation (explicit DFT sums, explicit phase
differences) and the closed form of the coherence dot product through
sums of unit phasors."""
import numpy as np
import pytest

from oracle import bold as B


def test_rest_is_a_fixed_point_with_zero_bold():
    Y, st = B.bold(np.zeros((3, 500)), 1.0, 10)
    assert np.all(Y == 0.0)
    assert np.array_equal(st, np.stack([np.zeros(3), np.ones(3), np.ones(3), np.ones(3)]))


def test_constant_drive_settles_on_the_closed_form_fixed_point():
    z = np.array([0.002, 0.005, 0.01])
    Y, st = B.bold(np.tile(z[:, None], (1, 12000)), 10.0, 100)    # 120 s at 10 ms
    for k in range(3):
        fp, y = B.bold_fixed_point(z[k])
        assert np.allclose(st[:, k], fp, rtol=1e-6, atol=1e-9)
        assert Y[k, -1] == pytest.approx(y, rel=1e-5)
    assert np.all(np.diff(Y[:, -1]) > 0)      # more drive, larger BOLD
    fp, y = B.bold_fixed_point(0.005)
    assert fp[1] > 1.0 and fp[2] > 1.0 and fp[3] < 1.0    # inflow and volume up, deoxyhaemoglobin down
    assert y > 0.0


def test_small_drives_respond_linearly_and_peak_a_few_seconds_after_a_pulse():
    T = 20000    # 20 s at 1 ms
    z = np.zeros(T)
    z[:100] = 1e-3    # a 0.1 s pulse
    Y1, _ = B.bold(z[None], 1.0, 10)
    Y2, _ = B.bold(2 * z[None], 1.0, 10)
    assert np.abs(Y2 - 2 * Y1).max() <= 1e-3 * np.abs(2 * Y1).max()
    t_peak = (np.argmax(Y1[0]) + 1) * 0.01
    assert 3.0 <= t_peak <= 7.0


def test_band_analytic_signal_of_an_in_band_sinusoid():
    T, tr = 400, 2.0
    t = np.arange(T) * tr
    f0 = 20 / (T * tr)        # 0.025 Hz, an exact bin in the band
    z = B.band_analytic(np.cos(2 * np.pi * f0 * t + 0.4)[None], tr)
    assert np.abs(z[0] - np.exp(1j * (2 * np.pi * f0 * t + 0.4))).max() < 1e-12
    z = B.band_analytic(np.cos(2 * np.pi * (120 / (T * tr)) * t)[None], tr)   # 0.15 Hz: out of band
    assert np.abs(z).max() < 1e-12


def test_phfcd_of_phase_locked_regions_is_one():
    T, tr = 300, 2.0
    t = np.arange(T) * tr
    f0 = 12 / (T * tr)
    Y = np.stack([np.cos(2 * np.pi * f0 * t + ph) for ph in (0.0, 0.5, 1.3, 2.0)])
    v, Tp = B.phfcd(Y, tr, discard=5)
    assert Tp == 300 - 10 and v.shape == (Tp * (Tp - 1) // 2,)
    assert np.allclose(v, 1.0, atol=1e-12)


def test_phfcd_against_brute_force_and_the_phasor_identity():
    rng = np.random.default_rng(3)
    N, T, tr, disc = 4, 30, 2.0, 2
    Y = rng.standard_normal((N, T)).cumsum(axis=1)
    got, Tp = B.phfcd(Y, tr, discard=disc, band=(0.01, 0.2))
    # brute force: explicit DFT sums, in-band positive bins doubled
    Yc = Y - Y.mean(axis=1, keepdims=True)
    z = np.zeros((N, T), dtype=complex)
    for k in range(N):
        F = [sum(Yc[k, s] * np.exp(-2j * np.pi * i * s / T) for s in range(T)) for i in range(T)]
        h = [2.0 if (0 < i < T / 2 and 0.01 <= i / (T * tr) <= 0.2) else 0.0 for i in range(T)]
        for s in range(T):
            z[k, s] = sum(F[i] * h[i] * np.exp(2j * np.pi * i * s / T) for i in range(T)) / T
    th = np.angle(z)[:, disc:T - disc]
    want = []
    for t1 in range(Tp):
        for t2 in range(t1 + 1, Tp):
            a = [np.cos(th[k, t1] - th[j, t1]) for k in range(N) for j in range(k + 1, N)]
            b = [np.cos(th[k, t2] - th[j, t2]) for k in range(N) for j in range(k + 1, N)]
            want.append(np.dot(a, b) / np.sqrt(np.dot(a, a) * np.dot(b, b)))
    assert np.allclose(got, want, atol=1e-12)
    # the coherence dot product through sums of unit phasors u_k:
    # V(t1).V(t2) = ((|sum u(t1) u(t2)|^2 - N) + (|sum u(t1) conj u(t2)|^2 - N)) / 4
    u = np.exp(1j * th)
    iu = np.triu_indices(N, k=1)
    for t1, t2 in ((0, 5), (3, 3), (7, 20)):
        v1 = np.cos(th[:, t1][:, None] - th[:, t1][None, :])[iu]
        v2 = np.cos(th[:, t2][:, None] - th[:, t2][None, :])[iu]
        A = (u[:, t1] * u[:, t2]).sum()
        Bc = (u[:, t1] * np.conj(u[:, t2])).sum()
        assert v1 @ v2 == pytest.approx(((abs(A) ** 2 - N) + (abs(Bc) ** 2 - N)) / 4, abs=1e-12)
