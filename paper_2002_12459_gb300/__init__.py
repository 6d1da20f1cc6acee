"""GB300-native join-project evaluation (two-path and star queries).

Importing this package loads nothing compiled.  ``paper_2002_12459_gb300.jp``
holds the Python binding of the C-ABI library ``libjp.so``; it fails loudly
when that library is missing.
"""
__all__ = ["workloads"]
