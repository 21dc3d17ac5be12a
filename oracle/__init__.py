"""CPU FP64 oracle of the FFT-accelerated BEM operator.

Test infrastructure: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline legs may import it.  See ``oracle.py``.
"""
