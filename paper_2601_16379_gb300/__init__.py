"""GB300-native k-ISDF fragment-ERI library (Python side).

The compute path lives in the C-ABI shared library built from ``csrc/``;
``binding`` marshals arguments to it.  ``workloads`` generates the seeded
synthetic inputs.  Importing the package does not load the library.
"""
__all__ = ["workloads", "binding"]
