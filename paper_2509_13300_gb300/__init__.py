"""GB300-native in-silico PCR hot path (AmpliconHunter, arXiv 2509.13300).

Scan degenerate primer sites on both strands with at most k mismatches, pair
them into amplicons inside a length window, and score each site's
nearest-neighbour melting temperature -- in hand-written sm_103a kernels
behind the C ABI declared in ``include/ampliconhunter.h``.

``paper_2509_13300_gb300.ah`` is the Python binding of that ABI (argument
marshalling only); ``paper_2509_13300_gb300.synth`` builds seeded synthetic
inputs.  Importing this package loads nothing native; the binding loads the
compiled library on first use and raises if it is missing.
"""
__all__ = ["ah", "synth"]
