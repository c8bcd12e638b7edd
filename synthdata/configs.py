"""The five workload configurations (sizes and parameters, no arithmetic).

Every number here is an input shared by both implementations.  Ring and
modulus parameters follow the RNS setting this project uses in place of the
paper's 64-bit torus (Table 2); WiSARD parameters follow the shape of the
paper's workloads (Table 3): address size, thermometer size and activation.

Field meanings
--------------
log_n        ring dimension N = 2^log_n of R = Z[X]/(X^N+1) (Section 2.1)
n_primes     number r of RNS primes q_i, Q = prod q_i
prime_bits   each q_i is below 2^prime_bits with q_i = 1 mod 2N
log_beta     gadget base beta = 2^log_beta; 0 means one digit per prime
             (beta = q_i, the RNS gadget)
log_p        plaintext modulus p = 2^log_p (Table 3 uses 2^8..2^13)
n_classes    l, number of discriminators
n_values     uint8 input values per sample (features or pixels)
therm_bits   thermometer width T per value (Section 2.3.2); s = n_values*T
tuple_bits   bits per RAM tuple before hashing
addr_bits    a, RAM address bits (= tuple_bits unless hashed)
hash_h3      1: each 16-bit tuple is H3-hashed to addr_bits on the client
act, act_arg PD-act activation: 'log', 'blog' (bound act_arg), 'bin' (thr)
"""
from dataclasses import dataclass, field, asdict


@dataclass(frozen=True)
class Config:
    name: str
    log_n: int
    n_primes: int
    prime_bits: int
    log_beta: int
    log_p: int
    n_classes: int
    n_values: int
    therm_bits: int
    tuple_bits: int
    addr_bits: int
    hash_h3: int
    act: str
    act_arg: int
    n_train: int
    n_test: int
    data_kind: str
    priors: tuple = field(default=())
    data_seed: int = 1
    model_seed: int = 7
    key_seed: int = 11

    def as_dict(self):
        return asdict(self)


CONFIGS = {
    # Plain method, tiny: Wisconsin-shaped (30 features, 2 classes).
    "cfg1": Config(name="cfg1", log_n=10, n_primes=1, prime_bits=30, log_beta=5,
                   log_p=8, n_classes=2, n_values=30, therm_bits=8, tuple_bits=8,
                   addr_bits=8, hash_h3=0, act="log", act_arg=0,
                   n_train=200, n_test=100, data_kind="gauss30",
                   priors=(0.5, 0.5)),
    # Batched: MNIST-shaped, 2-bit thermometer, 12-bit tuples.
    "cfg2": Config(name="cfg2", log_n=12, n_primes=2, prime_bits=50, log_beta=0,
                   log_p=16, n_classes=10, n_values=784, therm_bits=2, tuple_bits=12,
                   addr_bits=12, hash_h3=0, act="blog", act_arg=4,
                   n_train=1000, n_test=1000, data_kind="digits",
                   priors=(0.1,) * 10),
    # Batched at scale: 3-bit thermometer, 16-bit tuples H3-hashed to 12 bits.
    "cfg3": Config(name="cfg3", log_n=13, n_primes=3, prime_bits=55, log_beta=0,
                   log_p=20, n_classes=10, n_values=784, therm_bits=3, tuple_bits=16,
                   addr_bits=12, hash_h3=1, act="blog", act_arg=4,
                   n_train=60000, n_test=10000, data_kind="digits",
                   priors=(0.1,) * 10),
    # Batched skewed: HAM10000-shaped RGB, 7 classes with skewed priors.
    "cfg4": Config(name="cfg4", log_n=13, n_primes=3, prime_bits=55, log_beta=0,
                   log_p=22, n_classes=7, n_values=2352, therm_bits=3, tuple_bits=14,
                   addr_bits=14, hash_h3=0, act="bin", act_arg=1,
                   n_train=8012, n_test=2003, data_kind="lesions",
                   priors=(0.67, 0.11, 0.11, 0.05, 0.03, 0.02, 0.01)),
}


def get_config(cfg_name: str, **overrides) -> Config:
    """Return a named configuration, optionally with fields replaced."""
    cfg = CONFIGS[cfg_name]
    if overrides:
        d = cfg.as_dict()
        d.update(overrides)
        cfg = Config(**d)
    return cfg
