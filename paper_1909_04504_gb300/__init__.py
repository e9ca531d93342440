"""GB300-native WCSPH particle loop (PySPH paper, Sec. 2): CUDA kernels for sm_103a
behind the C ABI of ``include/sph.h``, with a thin ctypes binding."""
from .binding import (BatchSimulation, CONTINUITY, EDAC, DIAG_COUNT, DIAG_NAMES, FLUID, PREC_FP32, PREC_FP64,
                      INTEGRATOR_KDK, INTEGRATOR_PEC, CUBIC_SPLINE, final_kinetic_energy,
                      QUINTIC, STEP_GRAPH, STEP_PERSISTENT, SUMMATION, WALL, WALL_ADAMI, WALL_DENSITY,
                      WENDLAND_C2, Scheme, Simulation, SphError, VariableHSearch,
                      library_path, load, make_scheme, scheme_of)
from .build import build

__all__ = ["Simulation", "BatchSimulation", "VariableHSearch", "final_kinetic_energy", "Scheme", "SphError", "make_scheme", "scheme_of", "load", "build",
           "library_path", "QUINTIC", "WENDLAND_C2", "PREC_FP64", "PREC_FP32", "FLUID", "WALL",
           "CONTINUITY", "SUMMATION", "EDAC", "STEP_GRAPH", "STEP_PERSISTENT", "DIAG_COUNT", "DIAG_NAMES",
           "WALL_DENSITY", "WALL_ADAMI", "INTEGRATOR_KDK", "INTEGRATOR_PEC", "CUBIC_SPLINE"]
