"""Measurement code behind bench.py: the robustness sweep, the paper's own
workloads, the serving benchmark and the algorithmic-work tables of the
roofline.  Not part of the library: the package paper_2409_08729_gb300 never
imports it, and only these modules (never the library) may load the oracle
to check sampled outputs."""
