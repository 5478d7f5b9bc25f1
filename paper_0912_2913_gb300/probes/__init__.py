"""Hardware throughput probes (see run.py)."""
