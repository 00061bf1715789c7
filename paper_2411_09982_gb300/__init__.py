"""GB300 first-order Magnus time evolution: C-ABI CUDA library + thin binding.

`paper_2411_09982_gb300.magnus` loads `_lib/libmagnus.so` (built by
`paper_2411_09982_gb300.build`).  Importing the package does not load CUDA.
"""
