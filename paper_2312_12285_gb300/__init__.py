"""libpointsht: direct, pixel-free spherical-harmonic transform of weighted point
catalogs on GB300 (arXiv:2312.12285), exposed through a C ABI and a thin
Python binding.  See ``include/pointsht.h`` for the boundary."""
