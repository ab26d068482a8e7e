"""GB300 (sm_103a) particle-mesh forward model, adjoint, projected L-BFGS and
rank-order matching of MujicΛ, behind the C ABI in include/mujica_pm.h.

``api`` holds the Python binding (same names as the C entry points);
``inputs`` the seeded synthetic inputs; ``build`` compiles the library.
"""
__all__ = ["api", "inputs", "build"]
