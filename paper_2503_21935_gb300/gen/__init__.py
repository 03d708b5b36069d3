"""Process compiler: turns a process string into the op table ("program") that the
generic CUDA amplitude kernel executes, plus the exact colour matrix.

Sec. 2 of the paper describes per-process code generation (the CUDACPP plugin
generates the matrix-element code from the process); here the generated artefact
is a table of HELAS-style wavefunction, vertex, propagator and amplitude
operations rather than straight-line source, so one compiled kernel serves every
process.
"""
