"""GB300-native batched Matching-Pursuit encoder for adaptive quadtrees (AQMP).

The compute path is the C-ABI library ``libaqmp.so`` built from ``csrc/``;
``paper_2605_09190_gb300.aqmp`` is its thin ctypes binding.  Importing this
package loads nothing; the binding loads the library on first use and fails
loudly if it is missing.
"""
__all__ = ["aqmp", "synthetic"]
