"""Writes tests/golden/half_range_hermite_q200.txt: the half-range Gauss-Hermite
quadrature of order 200 (the HHLB(20;200) model of Sec. V) and its three-term
recurrence, from the oracle's mpmath construction (oracle/highorder.py) at
560 digits, rounded to 40.

    python tests/golden/make_half_range_tables.py [Q ...]

Calls only the oracle.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

from oracle import highorder  # noqa: E402

if __name__ == "__main__":
    for Q in [int(a) for a in sys.argv[1:]] or [200]:
        print(highorder.write_store(Q))
