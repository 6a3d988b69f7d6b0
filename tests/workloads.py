"""Seeded inputs for the tests: densities b built with the generator's
particles and the oracle's CIC and density preparation (so no input ever
comes from the code under test)."""
import numpy as np

from paper_1709_06350_gb300 import synth


def zeldovich_density(O, N, L, sigma_lin, R, seed):
    delta_L, dh = synth.linear_field(N, L, sigma_lin, seed)
    pos = synth.zeldovich_positions(dh, N, L)
    rho = O.cic_deposit(pos, N, L)
    return O.smooth_and_floor(rho, L, R), delta_L, pos


def smooth_density(N, seed, amp=0.6, kmax=2):
    b = 1.0 + synth.smooth_field(N, seed, amp, kmax=kmax)
    return np.maximum(b, 0.05) / np.maximum(b, 0.05).mean()
