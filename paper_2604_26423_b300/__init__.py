"""B300-native LR-QAOA state-vector simulation (arxiv 2604.26423, Sec. II-B).

The compute path is the CUDA library ``libqaoa.so`` (C ABI in ``include/qaoa.h``);
``paper_2604_26423_b300.qaoa`` is a thin ctypes binding over it and
``paper_2604_26423_b300.inputs`` draws seeded synthetic instances.
Importing this package loads nothing; the binding loads the library on first use.
"""
__all__ = ["inputs", "qaoa"]
