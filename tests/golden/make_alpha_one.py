"""Write alpha_one_d32.txt: inputs of a closed-form check of the estimator.

With the identity as P^-1 and every neighbour o_j = c + s_j for a sign
vector s_j in {-1,+1}^32, the normalized edge (o_j - c)/||o_j - c|| has all
coordinates +-1/sqrt(32), so it IS a codeword of Eq. (3): o_bar = o and
<o_bar, o> = 1.  The estimator <o_bar,q>/<o_bar,o> then equals <o,q>
exactly, and Eq. (2) returns the exact squared distance ||o_j - q||^2.
A query with integer coordinates spanning 0..15 is also reproduced exactly
by 4-bit quantization (v_l = 0, delta = 1).  So every estimate must equal
the integer ||o_j - q||^2 up to fp32 rounding.  Only numpy draws the
integers; the expected values are computed by the test from the vectors.
"""
import pathlib

import numpy as np

g = np.random.Generator(np.random.PCG64(20241119))
c = g.integers(-20, 21, size=32)
s = np.where(g.integers(0, 2, size=(32, 32)) == 1, 1, -1)
q = g.integers(0, 16, size=32)
q[3], q[17] = 0, 15  # span the full 4-bit range
out = pathlib.Path(__file__).with_name("alpha_one_d32.txt")
with open(out, "w") as f:
    f.write("# Closed-form estimator check (Sec. 2.2 Eq. (2)-(4), Sec. 3.1.1 Eq. (5)-(6)); see make_alpha_one.py\n")
    f.write("c " + " ".join(map(str, c)) + "\n")
    for j in range(32):
        f.write("s " + " ".join(map(str, s[j])) + "\n")
    f.write("q " + " ".join(map(str, q)) + "\n")
print(out)
