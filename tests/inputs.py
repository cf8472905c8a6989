"""Seeded test inputs: re-exported from the package's workload module, which holds
no arithmetic of the method (only seeds, sizes and raw random bytes)."""
from paper_1805_07339_b300.workloads import (HD, MASTER_SEED, TINY, hd_gather, random_indices,  # noqa: F401
                                             random_nv12)
