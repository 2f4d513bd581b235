"""GB300-native oversampling sample sort (SqDet / SqRan)."""
