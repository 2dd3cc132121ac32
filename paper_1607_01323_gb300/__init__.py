"""GB300-native matrix-free SIPG operators (arXiv:1607.01323): Python binding.

The binding is loaded lazily so that ``paper_1607_01323_gb300.inputs`` can be
imported on a machine without the built library.
"""
