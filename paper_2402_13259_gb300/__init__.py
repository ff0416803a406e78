"""GB300-native (sm_103a) Euler-approximation simulator for feedforward
Markovian queueing networks (Hong, Song & Wang, arXiv 2402.13259).

The compute path is the C-ABI library ``libeulernet.so`` built from
``csrc/``; ``binding`` marshals arguments to it.  Import ``binding`` lazily so
that the input generators in ``workloads`` stay importable on machines
without the CUDA library.
"""
__all__ = ["workloads", "binding"]
