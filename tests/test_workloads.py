"""The synthetic workloads are named by what they are; a name gives the same
seeded stream as the workload's seed offset."""

import numpy as np
import pytest

import workloads as W

NAMES = ["hodlr_n4096_m128_k8_r1_f64", "hss_n65536_m256_k32_r64", "hodlr_exp_n262144_m256_K8",
         "batched_512", "serving_64_hss"]


@pytest.mark.parametrize("name", NAMES)
def test_named_workloads_resolve(name):
    cfg = W.workload(name)
    assert cfg["name"] == name
    key = [k for k, v in W.CONFIGS.items() if v["name"] == name][0]
    a = W.rng_named(name, 3).standard_normal(5)
    b = W.rng_for(key, 3).standard_normal(5)
    assert np.array_equal(a, b)


def test_unknown_workload_rejected():
    with pytest.raises(KeyError):
        W.workload("no_such_workload")
    with pytest.raises(KeyError):
        W.rng_named("no_such_workload")
