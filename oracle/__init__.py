"""FP64 oracle of the SPIDER sampling step -- test infrastructure only.

Importable by `tests/`, `__graft_entry__.smoke()` and the CPU legs of
`bench.py`; never by the product path, which shares no code with it.
"""
from .spider_oracle import *  # noqa: F401,F403
