"""Seeded synthetic workloads shared by the CUDA path and the CPU oracle.

This package holds no arithmetic of the homomorphic WiSARD method: it only
names the five workload configurations and draws the raw uint8 input values
and labels that both implementations consume.  The paper's datasets
(Wisconsin, MNIST, HAM10000; Section 4.1) are not available, so these
generators stand in for them with the same shapes, class counts and priors.
"""
from .configs import CONFIGS, Config, get_config  # noqa: F401
from .gen import make_dataset  # noqa: F401
