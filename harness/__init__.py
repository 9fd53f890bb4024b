"""Seeded input generators shared by the oracle tests and the CUDA path.

`harness.tess` builds periodic Voronoi tessellations (a host-side C++
tessellator); `harness.ics` draws the synthetic initial conditions.  Nothing
here computes any step of the hydro update itself.
"""
