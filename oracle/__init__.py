"""The oracle: a plain single-threaded CPU Super Bloom filter.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2606_24417_gb300``) and never imports it.

``OracleSBF`` wraps ``sbf_oracle.c`` (Alg. 1 / Alg. 2 of the cuSBF paper, one
k-mer at a time); ``fpr`` holds the closed-form false-positive rates (Eq. 1,
Eq. 2 and their shard-aware forms).
"""
from .oracle import OracleSBF, build_oracle, oracle_library_path  # noqa: F401
