"""GB300-native EnSF analysis step (package root; the CUDA binding lives in
``paper_2407_12168_gb300.ensf`` and is loaded on first use)."""
