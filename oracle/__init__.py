"""The oracle: a plain, slow, FP64 CPU restatement of the sphere-GMRF sampler of
Creasey & Lang, arXiv 1709.10314.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) may import this
package.  The product path (``paper_1709_10314_gb300``) never imports it, and it never
imports the product path: the two share no code.

Parity status of each function is stated in ``oracle/oracle.py``.
"""
from .oracle import *  # noqa: F401,F403
