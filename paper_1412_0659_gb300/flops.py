"""The paper's flop convention for the tree force (Sec. VI.A).

Only force evaluation counts: one particle-particle interaction is 23 flops
(4 sub, 3 mul, 6 fma counted as 2, one rsqrt counted as 4) and one
particle-cell interaction with the quadrupole is 65 flops (4 sub, 6 add,
17 mul, 17 fma, one rsqrt).  Tree build, multipoles, the opening test,
integration and diagnostics count zero flops but do count in application
time.  The interaction counts are the ones recorded during execution.
"""

FLOPS_PP = 4 + 3 + 2 * 6 + 4          # = 23
FLOPS_PC = 4 + 6 + 17 + 2 * 17 + 4    # = 65


def tree_force_flops(n_pp: int, n_pc: int) -> float:
    """Flops of one force evaluation with n_pp p-p and n_pc p-c interactions."""
    return float(FLOPS_PP) * float(n_pp) + float(FLOPS_PC) * float(n_pc)


def fp32_peak_tflops(sm_count: int = 152, lanes_per_sm: int = 128, clock_mhz: float = 2070.0) -> float:
    """FP32 CUDA-core peak: SMs x FP32 lanes x 2 flops per FMA x clock."""
    return sm_count * lanes_per_sm * 2.0 * clock_mhz * 1e6 / 1e12
