"""Precision of one conv2d fused with StoC2 at 1024 channels per ciphertext (the single-conv
precision experiment of Sec. 6), on the CPU oracle.  The CUDA library computes the same limbs
(bit-exact parity), so the figure holds for both.

N = 2^16 on the config-2 chain, level 1 (Delta = 2^42), w = 8 (2l = 64 reals per slice, so
C = N / 2l = 1024 slices), 6 x 6 images with uniform [0, 1) pixels, C_in = C_out = C, 3 x 3
weights N(0, 0.1^2); the output is decrypted, decoded from the coefficient encoding and
compared with the FP64 conv2d.  Takes about four minutes on 16 host cores (building the
1024 fused diagonals dominates), so it is a script, not a test:

    python tests/precision_1024.py [channels]

Measured: MAE 3.7e-8, max 1.9e-7 at 1024 channels (the paper reports ~1.4e-6 for its own
library at 1024 channels per ciphertext).
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as WL  # noqa: E402
from oracle import encoding as E  # noqa: E402
from oracle.scheme import Oracle  # noqa: E402
from tests.pairs import oracle_params  # noqa: E402


def main(C=1024):
    P = oracle_params("cfg2")
    o = Oracle(P, 3)
    w0, w, f = 6, 8, 3
    slices = P.n // (w * w)
    assert C <= slices
    x = WL.image(3, C, w0)
    W = WL.weights(3, C, C, f, "normal")
    plan = o.conv_plan(W, C, C, f, w, 1, (2.0 ** 49 * float(P.q[1])) / P.delta[1])
    o.gen_rotation_keys(plan.rotations(P.n // 2))
    ct = o.encrypt(o.encode_pt(E.cins_input_slots(x, w, P.n), 1, P.delta[1]), 1)
    out = o.conv2d_cins(ct, plan)
    got = E.conv_output_from_coeffs(o.decode_coeffs(o.decrypt(out)), slices, w * w, C, w, w0)
    err = np.abs(got - E.conv2d_same(x, W))
    print("channels %d: MAE %.3g, max %.3g (%d PMult diagonals, %d rotations)"
          % (C, err.mean(), err.max(), len(plan.pts), len(plan.rotations(P.n // 2))))
    return err


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 1024)
