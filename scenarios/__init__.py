"""Seeded synthetic inputs for the polymer-flooding Newton step.

This package holds only input data generation (random fields, grid shapes,
well placement, schedules, physical constants). It contains none of the
method's arithmetic: no transmissibility, well index, property law or residual
term is computed here. Both the FP64 oracle (``oracle/``) and the CUDA path
(``paper_1807_05298_gb300``) read the same scenario dictionaries, so they see
bit-identical inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator, and normal deviates from the Box-Muller transform.
"""

from .generate import (  # noqa: F401
    splitmix64,
    uniform01,
    normal,
    default_physics,
    make_scenario,
    scenario_c1,
    scenario_c2,
    scenario_c3,
    scenario_member,
    scenario_1d_table1,
    scenario_2d_table2,
    scenario_layered_table4,
    scenario_size,
    DAY,
    BAR,
    MD,
    CP,
)
