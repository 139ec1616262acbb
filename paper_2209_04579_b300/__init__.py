"""B300-native key-sort-and-segment core of a tensor query processor.

Importing the package loads nothing native; ``paper_2209_04579_b300.tqp``
loads the CUDA library and raises if it is missing.
"""
