"""CPU FP64 oracle for the stencil / RK4 level path (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg import this
package; the product library never does.
"""
