"""Evaluation metrics of Sec. IV.

* pruning rate eta = 1 - d_G / d (Eq. pruning rate);
* first-round estimate eta_1 of Eq. (bound expectation) for a k-regular graph
  with J_hat ~ U(-alpha, alpha), h_hat ~ U(-beta, beta): the sum of k
  absolute couplings is replaced by a Gaussian with mean k alpha / 2 and
  variance k alpha^2 / 12, and eta_1 = P(b > a), b ~ U(0, beta);
* Hamiltonian ratio estimate chi_hat = 1/2 - E / (2 (sqrt(d) ||J||_F + ||h||_1))
  in the paper's (J, h) (Eq. hamiltonian ratio and the estimate after it);
* estimated time-to-solution T_TTS = T log(1 - 0.99) / log(1 - e^chi_hat / d)
  and speed v = chi_hat / T (Sec. IV-C).
"""

from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

from . import ising


def pruning_rate(d: int, d_g: int) -> float:
    return 1.0 - d_g / d


def eta1_estimate(k: int, alpha: float, beta: float) -> float:
    mean = k * alpha / 2.0
    sd = math.sqrt(k * alpha * alpha / 12.0)

    def cdf(x):
        return 0.5 * (1.0 + special.erf((x - mean) / (sd * math.sqrt(2.0))))

    val, _ = integrate.quad(lambda x: cdf(x) / beta, 0.0, beta, limit=200)
    return float(val)


def chi_hat(inst, E: float) -> float:
    A, b = ising.paper_form(inst)
    d = inst.n
    scale = math.sqrt(d) * float(np.linalg.norm(A)) + float(np.sum(np.abs(b)))
    return 0.5 - E / (2.0 * scale)


def tts(T: float, chi: float, d: int) -> float:
    return T * math.log(1.0 - 0.99) / math.log(1.0 - math.exp(chi) / d)


def speed(T: float, chi: float) -> float:
    return chi / T
