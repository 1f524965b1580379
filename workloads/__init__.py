"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package only *generates inputs*: graphs, Ising couplings and the dense site
tensors of the Ising tensor network (the paper's Sec. 7.1 construction).  It
contains none of the approximate-contraction method's arithmetic, so both the
CPU oracle and the CUDA path can consume its output without sharing code.
"""
