"""GB300-native CFR+ over games compiled to static dataflow.

``cfr`` is the thin binding of ``libcfr.so`` (C ABI in include/cfr.h);
``build`` compiles the library for sm_103a.
"""
