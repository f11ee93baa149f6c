"""Host helpers behind the bench's accuracy report: peak positions of a sampled
spectrum and the largest peak shift between two spectra."""
import numpy as np

from paper_1312_4698_gb300 import workloads as wl


def _lorentzians(E, centres, widths, heights):
    return sum(h * (0.5 * w) ** 2 / ((E - c) ** 2 + (0.5 * w) ** 2) for c, w, h in zip(centres, widths, heights))


def test_spectrum_peaks_recovers_line_centres():
    E = np.linspace(0.0, 100.0, 2001)                 # grid step 0.05
    centres = np.array([20.013, 47.5, 80.041])
    I = _lorentzians(E, centres, [2.0, 3.0, 2.5], [1.0, 0.3, 0.05])
    pk = wl.spectrum_peaks(E, I)
    assert pk.size == 3
    # the 3-point parabola on a grid 40x finer than the line width: well below the grid step
    assert np.max(np.abs(pk - centres)) < 2e-3


def test_spectrum_peaks_threshold_and_degenerate_input():
    E = np.linspace(0.0, 10.0, 101)
    I = _lorentzians(E, [3.0, 7.0], [0.5, 0.5], [1.0, 0.005])
    assert wl.spectrum_peaks(E, I).size == 1                  # the weak line is below 1 % of the maximum
    assert wl.spectrum_peaks(E, I, rel=0.001).size == 2
    assert wl.spectrum_peaks(E, np.full_like(I, np.nan)).size == 0
    assert wl.spectrum_peaks(E[:2], I[:2]).size == 0


def test_peak_shift():
    ref = np.array([1.0, 5.0, 9.0])
    assert wl.peak_shift(ref, ref) == 0.0
    assert abs(wl.peak_shift(ref, np.array([1.2, 4.9, 9.0, 20.0])) - 0.2) < 1e-12
    assert wl.peak_shift(ref, np.zeros(0)) == float("inf")
    assert wl.peak_shift(np.zeros(0), ref) == 0.0
