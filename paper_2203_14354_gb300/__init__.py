"""GB300-native Monte Carlo propagation of liquid-xenon scintillation photons
through a triangle-mesh detector (the optical simulation of a DARWIN-like
dual-phase TPC, arXiv:2203.14354).

* ``geometry``  -- procedural detector meshes, optical tables, photon sources
* ``tracker``   -- ``Tracker``: the CUDA library behind the C ABI of include/lxo.h
* ``calibrate`` -- gradient fit of optical parameters to per-PMT hit maps
* ``shard``     -- photon-id ranges per rank and the one tally reduction
* ``_capi``     -- ctypes binding with the C names
"""
from . import geometry  # noqa: F401

__all__ = ["geometry", "Tracker", "LightCollection", "EventLightCollection"]


def __getattr__(name):
    if name in ("Tracker", "LightCollection", "EventLightCollection"):
        from . import tracker
        return getattr(tracker, name)
    raise AttributeError(name)
