"""Seeded synthetic inputs (no transform arithmetic); see ``synth.fields``."""
from .fields import (cosine_mode, delta_field, draw_u64, energy_shape, seed_for_config,
                     signed_wavenumbers, spectral_velocity, splitmix64, uniform01, uniform_field)

__all__ = ["cosine_mode", "delta_field", "draw_u64", "energy_shape", "seed_for_config",
           "signed_wavenumbers", "spectral_velocity", "splitmix64", "uniform01", "uniform_field"]
