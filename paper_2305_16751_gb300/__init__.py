"""GB300-native (sm_103a) aggregation over dominated points.

``paper_2305_16751_gb300.domagg`` is the Python binding of the C library
(include/domagg.h); ``workloads`` draws the seeded synthetic inputs.
"""
