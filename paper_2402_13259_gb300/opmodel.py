"""Algorithmic operation count of one Euler unit (one station, one
replication, one step), for the ALU roofline.

The Euler step is integer state updated by float32 samplers: no dense
contraction, negligible memory traffic (the state lives in shared memory),
so the binding resource is the SM's instruction issue (FP32/INT32 lanes).
The count below is the number of arithmetic operations (integer or float
add/mul/fma/compare/select/shift/logic/convert, IEEE division and square
root counted as one each) that the sampler definitions of this library
perform per event, counted from the source; loads, stores, moves and
branches are not counted.  Multiplied by event frequencies measured on a
sample of the workload it gives algorithmic operations per unit; divided by
the kernel's time it gives achieved operations per second, compared with the
SM issue peak (SMs x 128 lanes x clock).
"""
from __future__ import annotations

from typing import Dict

# operations per elementary function call
EXP = 22      # 2 range tests, mul+add+floor, 2 fma reduction, 8 fma, cvt+shift+add, mul
LOG = 26      # 4 special tests, exponent split (shift, sub, and, or), compare+scale, sub,
              # add+div, mul, 4 fma, mul, mul, fma, add, cvt, 2 fma
EXPM1 = 12    # abs+compare, 7 fma, mul, fma
LOG1P = 4 + LOG
STIRLING_SMALL = 3 + LOG + 4 + 9 + LOG  # (k+.5) log k - k + c; small factorial product + log
STIRLING_SERIES = 6
BD0_SERIES = 6 + 5 * 3                # setup (sub, abs, add, mul, compare, div...), 5 terms
LOGPMF_POIS = 2 + LOG + 2 + STIRLING_SERIES + BD0_SERIES
LOGPMF_BINOM = 3 * STIRLING_SERIES + 2 * BD0_SERIES + 2 * LOG + LOG1P + 8
# constants of a binomial's p (symmetry test and flip, q = 1 - p, r = p/q,
# ln(1 - p)): per draw only where p varies (Algorithm 1's x > m branches); the
# per-station p0 and the per-edge routing probabilities have them precomputed
BINOM_CONST = 6 + LOG1P

COST: Dict[str, float] = {
    # per event counted by the oracle's work counters
    "philox_blocks": 10 * 10 + 2,      # 10 rounds x (2 mul.lo, 2 mul.hi, 4 xor, 2 key adds)
    "uniforms": 5,                     # shift, shift, or, convert, scale
    "pois_inv": EXP + 3,
    "pois_inv_iters": 6,               # mul, mul, add, compare x2, increment
    "pois_ptrs": 14,                   # sqrt, 6 mul/add, 2 div, 2 sub
    "pois_ptrs_iters": 14,             # 2 sub, abs, div, 2 fma-like, floor, 4 compares
    "pois_ptrs_logtests": LOG + 5 + LOGPMF_POIS,
    "bin_inv": EXP + 8,                # (1 - p)^n = exp(n ln(1 - p)), F, u, loop set-up
    "bin_inv_iters": 7,
    "bin_btrs": 20 + LOGPMF_BINOM,
    "bin_btrs_iters": 14,
    "bin_btrs_logtests": LOG + 5 + LOGPMF_BINOM + 1,
    "gamma_small": 3,
    "gamma_small_logs": LOG + 4,
    "gamma_mt": 6,
    "gamma_mt_iters": 14 + 0.05 * (2 * LOG + 8),  # squeeze accepts ~95 %
    "normal_iters": 8 + 0.785 * (LOG + 4),
    "dep_le_m": 2,
    "dep_t_gt_h": 4 + BINOM_CONST,
    "dep_t_le_h": 6 + EXPM1 + BINOM_CONST,
    "route_binomials": 3,
    "gather_edges": 2,
    "units": 24,                       # stream keys, state update, overflow test, 5 statistics
}


def ops_per_unit(counters: Dict[str, int]) -> float:
    units = max(counters.get("units", 0), 1)
    total = sum(COST[k] * counters.get(k, 0) for k in COST)
    return total / units
