"""The roofline numerator: the algorithmic FP64 operation count of the integrator
(paper_2312_13513_gb300/flops.py) against counts it cannot exceed or must equal.

* Upper bound: for the same sub-step history, the model's flops and transcendentals never exceed
  what the plain dense oracle executes (its op-counting scalar type counts every add, mul, div,
  sqrt, exp, log and pow; a multiply-add there is two operations, as in the model).  A model that
  counted work the algorithm does not do would inflate the reported roofline fraction.
* Exact terms: the dense LU with partial pivoting and the two triangular solves have textbook
  operation counts, sum_k ((N-k-1) + 2 (N-k-1)^2) = 2N^3/3 - N^2/2 - N/6 (plus N pivot
  reciprocals) and 2N^2 - N.
"""
import numpy as np
import pytest

import oracle
from paper_2312_13513_gb300 import flops as fl

from helpers import random_states


@pytest.mark.parametrize("which,fuel", [("h2", "H2"), ("ch4", "CH4")])
def test_model_never_exceeds_the_executed_operations(which, fuel, request):
    om = request.getfixturevalue("om_" + which)
    mech = om.mech
    T, p, Y = random_states(mech, 3, 2, fuel)
    for i in range(T.size):
        c, st, nsub, nrej = om.count_ops(p[i], np.r_[T[i], Y[:, i]], 1e-6)
        assert st == oracle.OK and nsub > 0
        executed = c["add"] + c["mul"] + c["div"] + c["sqrt"]
        executed_tr = c["exp"] + c["log"] + c["pow"]
        flops, trans, _ = fl.launch_flops(mech, nsub, nsub + nrej)
        assert 0.1 * executed < flops <= executed, (flops, executed)
        assert 0.1 * executed_tr < trans <= executed_tr, (trans, executed_tr)


@pytest.mark.parametrize("N", [2, 10, 54])
def test_dense_lu_and_solve_counts_are_the_textbook_ones(N):
    assert 6 * (fl.lu_flops(N) - N) == 4 * N ** 3 - 3 * N ** 2 - N     # 2N^3/3 - N^2/2 - N/6
    assert fl.solve_flops(N) == N * (N - 1) + N * (N - 1) + N          # two substitutions, N divisions
