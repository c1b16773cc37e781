"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds random draws and workload definitions only: no step of the
method's arithmetic (no Hamiltonian construction, no filter, no Lanczos).
Every random number comes from SplitMix64 (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), used in counter form:
the i-th output of a stream seeded with ``seed`` is ``mix64(seed + (i+1)*G)``
with G = 0x9E3779B97F4A7C15.
"""
from .rng import splitmix64, uniform01, uniform_pm_half, normals
from .workloads import (XXZParams, QSunParams, HubbardParams, QREMParams, xxz_params, qsun_params,
                        hubbard_params, qrem_params, j1j2_params, xxz_flux_params, qsun_u1_params, CONFIGS, config_seed, serving_stream,
                        PBC, OBC)

__all__ = ["splitmix64", "uniform01", "uniform_pm_half", "normals", "XXZParams",
           "QSunParams", "HubbardParams", "QREMParams", "xxz_params", "qsun_params", "hubbard_params",
           "qrem_params", "j1j2_params", "xxz_flux_params", "qsun_u1_params", "CONFIGS", "config_seed", "serving_stream", "PBC", "OBC"]
