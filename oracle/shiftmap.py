"""Fitted shift-exponent map of Sec. 5 (eq. shiftexp, Table tab:optweights).

TEST INFRASTRUCTURE (see oracle/__init__.py).

sigma_p(k, l) = clamp(2 - exp(-alpha(l) (k - k_c(l))), 1, 2) with
k_c(l) = kc1 exp(kc0 l), alpha(l) = a1 exp(a0 l), h = 2^-l; the shift is
epsilon = k^sigma. The weights are those the paper prints for Q_p elements.
"""
import math

# (kc0, kc1, a0, a1) per order p, as printed in Table tab:optweights.
PAPER_WEIGHTS = {
    1: (0.4592788619853418, 2.5790032999702346, -0.6261637288068426, 1.7580549857142198),
    2: (0.5736926870738827, 2.5729974893966001, -0.6615199737374460, 1.5966386518185063),
    3: (0.6305770719029798, 2.4284320222555804, -0.4465407372367102, 0.1287828338493968),
}


def sigma(k, level, weights):
    kc0, kc1, a0, a1 = weights
    kc = kc1 * math.exp(kc0 * level)
    alpha = a1 * math.exp(a0 * level)
    beta = 2.0 - math.exp(-alpha * (k - kc))
    return min(max(beta, 1.0), 2.0)


def shift(k, level, weights):
    return k ** sigma(k, level, weights)
