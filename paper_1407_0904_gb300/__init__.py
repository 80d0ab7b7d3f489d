"""GB300 finite-element local assembly (COFFEE, arXiv:1407.0904): Python binding.

The compute path is libcoffee.so (hand-written CUDA for sm_103a behind the C ABI in
include/coffee.h); ``binding`` marshals torch tensors into it. ``meshgen`` holds the
seeded synthetic input generators.
"""
from .binding import *  # noqa: F401,F403
from .binding import lib, CoffeeError  # noqa: F401
