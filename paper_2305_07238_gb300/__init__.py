"""Progressive Material Caching (Fujieda & Harada 2022) on GB300 (sm_103a).

The compute path is the C-ABI library ``libpmc.so`` built from ``csrc/``; the Python
binding in :mod:`paper_2305_07238_gb300.pmc` only marshals arguments into it.
Importing the package does not load the library; the first call into the binding
does, and fails loudly if it is missing.
"""
