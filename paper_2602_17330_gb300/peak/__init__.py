"""Issue-rate microbenchmark behind the alignment kernel's integer roofline.

``python -m paper_2602_17330_gb300.peak`` compiles alu_peak.cu for sm_103a and
prints lane-operations per SM per clock for the operations the alignment
recurrence uses (3-input add, max, DPX max3/add-max with relu in 32-bit and
packed 16-bit form, multiply-add, FP32 max).
"""
