"""Seeded synthetic inputs (CNN-shaped), shared by the tests, smoke() and bench.py.

This module only draws numbers: no encoding, no modular arithmetic, nothing of the
method.  Both the oracle and the CUDA library receive the same arrays from here.

Stand-ins for the paper's data (CIFAR / ImageNet images and trained weights are
not available): pixels uniform in [0, 1), conv weights uniform[-1, 1] (config 1)
or Gaussian (config 2: sigma 0.1).
"""
import numpy as np

# ring / chain shapes, one dict per named configuration
PARAMS = {
    # N = 2^12, 6 primes: q0 60-bit, 3 x 40-bit scaling, 2 x 60-bit special, dnum = 2, scale 2^40
    "cfg1": dict(log_n=12, n_q=4, dnum=2, n_p=0, q0_bits=60, scale_bits=40, p_bits=60, boot_bits=0, n_boot=0,
                 h=0, sigma=3.2),
    # N = 2^16, 24 Q-limbs (9 circuit levels at 2^42, 14 bootstrapping levels at 2^48), dnum = 3,
    # 7 special 60-bit primes, h = 192
    "cfg2": dict(log_n=16, n_q=24, dnum=3, n_p=7, q0_bits=60, scale_bits=42, p_bits=60, boot_bits=48, n_boot=14,
                 h=192, sigma=3.2),
    # the config-2 chain at N = 2^10 (small enough for the CPU oracle to run a whole block)
    "cfg2_small": dict(log_n=10, n_q=24, dnum=3, n_p=7, q0_bits=60, scale_bits=42, p_bits=60, boot_bits=48,
                       n_boot=14, h=192, sigma=3.2),
}

CONV = {
    "cfg1": dict(cin=1, cout=1, w0=16, f=3, weight="uniform"),
    "cfg2": dict(cin=16, cout=16, w0=32, f=3, weight="gauss"),
    "cfg2_small": dict(cin=4, cout=4, w0=4, f=3, weight="gauss"),
    # the stride-1 block shapes of the three stages of a ResNet-20-shaped network (config 3)
    "cfg3_s1": dict(cin=16, cout=16, w0=32, f=3, weight="gauss"),
    "cfg3_s2": dict(cin=32, cout=32, w0=16, f=3, weight="gauss"),
    "cfg3_s3": dict(cin=64, cout=64, w0=8, f=3, weight="gauss"),
}


def image(seed, cin, w0):
    """input feature map (cin, w0, w0), uniform [0, 1)"""
    return np.random.default_rng(seed).random((cin, w0, w0))


def weights(seed, cout, cin, f, kind):
    """conv weights (cout, cin, f, f): uniform[-1, 1] or N(0, 0.1^2)"""
    rng = np.random.default_rng(seed + 7919)
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, (cout, cin, f, f))
    return rng.normal(0.0, 0.1, (cout, cin, f, f))


def residues(seed, moduli, n):
    """uniform residues, one row per modulus (for raw kernel tests)"""
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, int(q), size=n, dtype=np.uint64) for q in moduli])


def slots(seed, m, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * (rng.normal(size=m) + 1j * rng.normal(size=m))
