"""CPU FP64 oracle of the moving-mesh MUSCL-Hancock update.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline leg of bench.py, never by the CUDA path.
"""
