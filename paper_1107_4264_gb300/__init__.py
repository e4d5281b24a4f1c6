"""GB300-native X-engine (per-channel cross-correlation of station voltages).

The native library is loaded on first use by :mod:`paper_1107_4264_gb300.xc`.
"""
